"""ctypes binding of the C ABI declared in include/lbm.h.

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions keep the ABI's names; ``Solver`` bundles a handle
with numpy-array helpers.  There is no fallback: if ``liblbm.so`` is missing
or the GPU is absent, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, EREACH, ETIMEOUT, EBUDGET = range(8)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
                4: "LBM_ESTATE", 5: "LBM_EREACH", 6: "LBM_ETIMEOUT",
                7: "LBM_EBUDGET"}
F32, F64 = 0, 1
TRANSMISSIVE, REFLECTING, PERIODIC = 0, 1, 2
PLANAR_X, CIRCLE = 0, 1


class lbm_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("gamma", ctypes.c_double),
                ("theta", ctypes.c_double), ("dt", ctypes.c_double),
                ("max_reach", ctypes.c_int32), ("kahan", ctypes.c_int32),
                ("cons_every", ctypes.c_int32), ("reserved_", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class lbm_prim(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("u", ctypes.c_double),
                ("v", ctypes.c_double), ("p", ctypes.c_double)]


class lbm_noalloc_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("gamma", ctypes.c_double), ("theta", ctypes.c_double)]


class lbm_tube(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nsteps", ctypes.c_int64),
                ("dt", ctypes.c_double), ("x_d", ctypes.c_double),
                ("left", lbm_prim), ("right", lbm_prim),
                ("bc", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class lbm_grid2d(ctypes.Structure):
    _fields_ = [("cfg", lbm_config), ("inner", lbm_prim), ("outer", lbm_prim),
                ("geom", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("a0", ctypes.c_double), ("a1", ctypes.c_double),
                ("radius", ctypes.c_double), ("nsteps", ctypes.c_int64)]


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_DP = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p


def load() -> ctypes.CDLL:
    """Load liblbm.so (built by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "lbm_abi_version": ([], ctypes.c_int32),
        "lbm_create": ([ctypes.POINTER(lbm_config), ctypes.POINTER(_H)], ctypes.c_int),
        "lbm_init_riemann": ([_H, ctypes.POINTER(lbm_prim), ctypes.POINTER(lbm_prim),
                              ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double], ctypes.c_int),
        "lbm_set_primitives": ([_H, _DP, _DP, _DP, _DP, ctypes.c_int64], ctypes.c_int),
        "lbm_set_moments": ([_H, _DP, _DP, _DP, _DP, ctypes.c_int64], ctypes.c_int),
        "lbm_step": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_moments": ([_H, _DP, _DP, _DP, _DP, _DP, ctypes.c_int64], ctypes.c_int),
        "lbm_conservation": ([_H, _DP], ctypes.c_int),
        "lbm_last_totals": ([_H, _DP], ctypes.c_int),
        "lbm_reach": ([_H, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "lbm_diagnostics": ([_H, ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        "lbm_synchronize": ([_H], ctypes.c_int),
        "lbm_lambda": ([_H], ctypes.c_double),
        "lbm_last_error": ([_H], ctypes.c_char_p),
        "lbm_destroy": ([_H], None),
        "lbm_batch_create": ([ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int32, ctypes.POINTER(lbm_tube),
                              ctypes.c_int64, ctypes.c_void_p,
                              ctypes.POINTER(_H)], ctypes.c_int),
        "lbm_batch_run": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_batch_sync": ([_H, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
        "lbm_batch_moments": ([_H, ctypes.c_int64, _DP, _DP, _DP, _DP,
                               ctypes.c_int64], ctypes.c_int),
        "lbm_batch_totals": ([_H, _DP, ctypes.c_int64], ctypes.c_int),
        "lbm_batch_last_error": ([_H], ctypes.c_char_p),
        "lbm_batch_destroy": ([_H], None),
        "lbm_pool_create": ([ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                             ctypes.c_void_p, ctypes.POINTER(_H)], ctypes.c_int),
        "lbm_pool_add": ([_H, ctypes.POINTER(lbm_tube),
                          ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "lbm_pool_step": ([_H], ctypes.c_int),
        "lbm_pool_run": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_pool_progress": ([_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "lbm_pool_read": ([_H, ctypes.c_int32, _DP, _DP, _DP, _DP,
                           ctypes.c_int64], ctypes.c_int),
        "lbm_pool_remove": ([_H, ctypes.c_int32], ctypes.c_int),
        "lbm_pool_last_error": ([_H], ctypes.c_char_p),
        "lbm_pool_destroy": ([_H], None),
        "lbm_measure_fma_peak": ([ctypes.c_int32, _DP, ctypes.c_void_p],
                                 ctypes.c_int),
        "lbm_check_fp32_arith": ([ctypes.c_int64, ctypes.c_uint64, _DP,
                                  ctypes.c_void_p], ctypes.c_int),
        "lbm_batch_tuning": ([_H, ctypes.POINTER(ctypes.c_int32), _DP],
                             ctypes.c_int),
        "lbm_batch_set_tile": ([_H, ctypes.c_int32], ctypes.c_int),
        "lbm_batch2d_create": ([ctypes.POINTER(lbm_grid2d), ctypes.c_int32,
                                ctypes.c_void_p, ctypes.POINTER(_H)],
                               ctypes.c_int),
        "lbm_batch2d_run": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_batch2d_steps": ([_H, ctypes.POINTER(ctypes.c_int64)],
                              ctypes.c_int),
        "lbm_batch2d_moments": ([_H, ctypes.c_int32, _DP, _DP, _DP, _DP, _DP,
                                 ctypes.c_int64], ctypes.c_int),
        "lbm_batch2d_last_error": ([_H], ctypes.c_char_p),
        "lbm_batch2d_destroy": ([_H], None),
        "lbm_bgk_create": ([ctypes.POINTER(lbm_config), ctypes.c_double,
                            ctypes.POINTER(_H)], ctypes.c_int),
        "lbm_bgk_init_riemann": ([_H, ctypes.POINTER(lbm_prim),
                                  ctypes.POINTER(lbm_prim), ctypes.c_int32,
                                  ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double], ctypes.c_int),
        "lbm_bgk_set_moments": ([_H, _DP, _DP, _DP, _DP, ctypes.c_int64],
                                ctypes.c_int),
        "lbm_bgk_set_packets": ([_H, _DP, ctypes.c_int64], ctypes.c_int),
        "lbm_bgk_packets": ([_H, _DP, ctypes.c_int64], ctypes.c_int),
        "lbm_bgk_step": ([_H, ctypes.c_int64], ctypes.c_int),
        "lbm_bgk_moments": ([_H, _DP, _DP, _DP, _DP, _DP, ctypes.c_int64],
                            ctypes.c_int),
        "lbm_bgk_conservation": ([_H, _DP], ctypes.c_int),
        "lbm_bgk_diagnostics": ([_H, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_uint32)],
                                ctypes.c_int),
        "lbm_bgk_synchronize": ([_H], ctypes.c_int),
        "lbm_bgk_last_error": ([_H], ctypes.c_char_p),
        "lbm_bgk_destroy": ([_H], None),
        "lbm_step_noalloc": ([ctypes.POINTER(lbm_noalloc_desc),
                              ctypes.c_void_p * 4, ctypes.c_void_p * 4,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t],
                             ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


def _f64(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"array of {a.size} values, expected {n}")
    return a


def _check(h, st):
    if st != OK:
        msg = load().lbm_last_error(h)
        raise LbmError(st, msg.decode() if msg else "")


def make_config(dim, nx, ny=1, *, x0=0.0, x1=1.0, y0=0.0, gamma=1.4,
                theta=None, dt=None, precision=F64, bc_x=TRANSMISSIVE,
                bc_y=REFLECTING, max_reach=0, kahan=1, cons_every=0,
                stream=None) -> lbm_config:
    """lbm_config with the defaults of the Sod problem (Section V.C)."""
    dx = (x1 - x0) / nx
    if theta is None:
        theta = 0.5 if dim == 1 else 0.0
    return lbm_config(dim, precision, bc_x, bc_y, nx, ny if dim == 2 else 1,
                      x0, x1, y0, gamma, theta, dx if dt is None else dt,
                      max_reach, kahan, cons_every, 0, stream)


class Solver:
    """One handle of the C ABI."""

    def __init__(self, cfg: lbm_config):
        lib = load()
        self.cfg = cfg
        self.n = cfg.nx * cfg.ny
        self.dim = cfg.dim
        h = _H()
        st = lib.lbm_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise LbmError(st, "lbm_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().lbm_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def lam(self) -> float:
        return load().lbm_lambda(self.h)

    def init_riemann(self, inner, outer, geom=PLANAR_X, a0=0.5, a1=0.5,
                     radius=0.0):
        """inner/outer: (rho, u, p) or (rho, u, v, p)."""
        def prim(s):
            s = tuple(float(v) for v in s)
            return lbm_prim(*(s if len(s) == 4 else (s[0], s[1], 0.0, s[2])))
        a, b = prim(inner), prim(outer)
        _check(self.h, load().lbm_init_riemann(self.h, ctypes.byref(a),
                                               ctypes.byref(b), geom, a0, a1,
                                               radius))

    def set_primitives(self, rho, u, v, p):
        n = self.n
        rho, u, v, p = (_f64(x, n) for x in (rho, u, v, p))
        _check(self.h, load().lbm_set_primitives(self.h, _dp(rho), _dp(u),
                                                 _dp(v), _dp(p), n))

    def set_moments(self, rho, mx, my, rhoE):
        n = self.n
        rho, mx, my, rhoE = (_f64(x, n) for x in (rho, mx, my, rhoE))
        _check(self.h, load().lbm_set_moments(self.h, _dp(rho), _dp(mx),
                                              _dp(my), _dp(rhoE), n))

    def step(self, nsteps=1):
        _check(self.h, load().lbm_step(self.h, int(nsteps)))

    def moments(self, out=None) -> dict:
        """Physical rho, mx, my (2-D), rhoE, p as float64 arrays."""
        n = self.n
        if out is None:
            out = {k: np.empty(n) for k in ("rho", "mx", "rhoE", "p")}
            if self.dim == 2:
                out["my"] = np.empty(n)
        _check(self.h, load().lbm_moments(
            self.h, _dp(out["rho"]), _dp(out["mx"]), _dp(out.get("my")),
            _dp(out["rhoE"]), _dp(out.get("p")), n))
        return out

    def conservation(self) -> np.ndarray:
        out = np.zeros(4)
        _check(self.h, load().lbm_conservation(self.h, _dp(out)))
        return out

    def last_totals(self) -> np.ndarray:
        """Totals the step kernel formed at the last summing step."""
        out = np.zeros(4)
        _check(self.h, load().lbm_last_totals(self.h, _dp(out)))
        return out

    def reach(self) -> int:
        r = ctypes.c_int32(0)
        _check(self.h, load().lbm_reach(self.h, ctypes.byref(r)))
        return r.value

    def diagnostics(self) -> dict:
        s, e, f = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_uint32(0)
        _check(self.h, load().lbm_diagnostics(self.h, ctypes.byref(s),
                                              ctypes.byref(e), ctypes.byref(f)))
        return {"steps": s.value, "eclamps": e.value, "flags": f.value}

    def synchronize(self):
        _check(self.h, load().lbm_synchronize(self.h))


class Bgk:
    """One relaxation-time (tau != 1, eqs 4-5) handle of the C ABI: the
    state is per packet, shaped (slots, fields, nodes) at this binding
    (slots 5 / 8, fields dim + 2), physical units."""

    def __init__(self, cfg: lbm_config, tau: float):
        lib = load()
        self.cfg = cfg
        self.n = cfg.nx * cfg.ny
        self.dim = cfg.dim
        self.slots = 5 if cfg.dim == 1 else 8
        self.fields = cfg.dim + 2
        h = _H()
        st = lib.lbm_bgk_create(ctypes.byref(cfg), float(tau), ctypes.byref(h))
        if st != OK:
            raise LbmError(st, "lbm_bgk_create")
        self.h = h

    def _check(self, st):
        if st != OK:
            msg = load().lbm_bgk_last_error(self.h)
            raise LbmError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            load().lbm_bgk_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_riemann(self, inner, outer, geom=PLANAR_X, a0=0.5, a1=0.5,
                     radius=0.0):
        a, b = lbm_prim(*_prim4(inner)), lbm_prim(*_prim4(outer))
        self._check(load().lbm_bgk_init_riemann(self.h, ctypes.byref(a),
                                                ctypes.byref(b), geom, a0, a1,
                                                radius))

    def set_moments(self, rho, mx, my, rhoE):
        n = self.n
        rho, mx, my, rhoE = (_f64(x, n) for x in (rho, mx, my, rhoE))
        self._check(load().lbm_bgk_set_moments(self.h, _dp(rho), _dp(mx),
                                               _dp(my), _dp(rhoE), n))

    def set_packets(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (self.slots, self.fields, self.n):
            raise ValueError(f"packets of shape {f.shape}")
        self._check(load().lbm_bgk_set_packets(self.h, _dp(f), self.n))

    def packets(self) -> np.ndarray:
        f = np.empty((self.slots, self.fields, self.n))
        self._check(load().lbm_bgk_packets(self.h, _dp(f), self.n))
        return f

    def step(self, nsteps=1):
        self._check(load().lbm_bgk_step(self.h, int(nsteps)))

    def moments(self) -> dict:
        n = self.n
        out = {k: np.empty(n) for k in ("rho", "mx", "rhoE", "p")}
        if self.dim == 2:
            out["my"] = np.empty(n)
        self._check(load().lbm_bgk_moments(
            self.h, _dp(out["rho"]), _dp(out["mx"]), _dp(out.get("my")),
            _dp(out["rhoE"]), _dp(out["p"]), n))
        return out

    def conservation(self) -> np.ndarray:
        out = np.zeros(4)
        self._check(load().lbm_bgk_conservation(self.h, _dp(out)))
        return out

    def diagnostics(self) -> dict:
        s, e = ctypes.c_int64(0), ctypes.c_int64(0)
        r, f = ctypes.c_int32(0), ctypes.c_uint32(0)
        self._check(load().lbm_bgk_diagnostics(self.h, ctypes.byref(s),
                                               ctypes.byref(e), ctypes.byref(r),
                                               ctypes.byref(f)))
        return {"steps": s.value, "eclamps": e.value, "reach": r.value,
                "flags": f.value}

    def synchronize(self):
        self._check(load().lbm_bgk_synchronize(self.h))


def lbm_step_noalloc(desc: lbm_noalloc_desc, inputs, outputs, totals=0,
                     reach=0, flags=0, stream=0) -> None:
    """One step between caller-owned device arrays (integer device
    addresses, order rho, m_x, m_y, rhoE; 0 for m_y in 1-D) without any
    allocation by the library.  Raises LbmError with the library's message."""
    lib = load()
    ins = (ctypes.c_void_p * 4)(*[a or None for a in inputs])
    outs = (ctypes.c_void_p * 4)(*[a or None for a in outputs])
    err = ctypes.create_string_buffer(512)
    st = lib.lbm_step_noalloc(ctypes.byref(desc), ins, outs, totals or None,
                              reach or None, flags or None, stream or None,
                              err, len(err))
    if st != OK:
        raise LbmError(st, err.value.decode())


def lbm_measure_fma_peak(precision, stream=None) -> float:
    """Fused multiply-add throughput (flop/s) of the current device in
    precision F32 or F64 (measurement; see include/lbm.h)."""
    out = ctypes.c_double(0.0)
    st = load().lbm_measure_fma_peak(int(precision), ctypes.byref(out),
                                     stream)
    if st != OK:
        raise LbmError(st, "lbm_measure_fma_peak")
    return out.value


def lbm_check_fp32_arith(n, seed=1, stream=None) -> tuple[float, float]:
    """Largest ulp distances of the FP32 kernels' reciprocal and quotient
    from CUDA's correctly rounded division over n generated inputs
    (diagnostics; see include/lbm.h)."""
    out = (ctypes.c_double * 2)()
    st = load().lbm_check_fp32_arith(int(n), int(seed), out, stream)
    if st != OK:
        raise LbmError(st, "lbm_check_fp32_arith")
    return out[0], out[1]


def make_tube(n, nsteps, dt, left, right, x_d=0.5, bc=TRANSMISSIVE) -> lbm_tube:
    """left/right: (rho, u, p)."""
    L_ = lbm_prim(float(left[0]), float(left[1]), 0.0, float(left[2]))
    R_ = lbm_prim(float(right[0]), float(right[1]), 0.0, float(right[2]))
    return lbm_tube(int(n), int(nsteps), float(dt), float(x_d), L_, R_, bc, 0)


class Batch:
    """Many independent 1-D tubes advanced together (lbm_batch_*)."""

    def __init__(self, tubes, precision=F32, gamma=1.4, theta=0.5, kahan=1,
                 stream=None):
        lib = load()
        arr = (lbm_tube * len(tubes))(*tubes)
        self.tubes = list(tubes)
        h = _H()
        st = lib.lbm_batch_create(precision, gamma, theta, kahan, arr,
                                  len(tubes), stream, ctypes.byref(h))
        if st != OK:
            raise LbmError(st, "lbm_batch_create")
        self.h = h

    def _check(self, st):
        if st != OK:
            msg = load().lbm_batch_last_error(self.h)
            raise LbmError(st, msg.decode() if msg else "")

    def run(self, max_launches=-1):
        self._check(load().lbm_batch_run(self.h, int(max_launches)))

    def sync(self):
        s, f = ctypes.c_int64(0), ctypes.c_uint32(0)
        self._check(load().lbm_batch_sync(self.h, ctypes.byref(s),
                                          ctypes.byref(f)))
        return s.value

    def moments(self, j) -> dict:
        n = self.tubes[j].n
        out = {k: np.empty(n) for k in ("rho", "mx", "rhoE", "p")}
        self._check(load().lbm_batch_moments(
            self.h, j, _dp(out["rho"]), _dp(out["mx"]), _dp(out["rhoE"]),
            _dp(out["p"]), n))
        return out

    def totals(self) -> np.ndarray:
        out = np.zeros(3 * len(self.tubes))
        self._check(load().lbm_batch_totals(self.h, _dp(out), len(self.tubes)))
        return out.reshape(-1, 3)

    def tuning(self) -> dict:
        """Tile width in use and measured ms per step of 128, 256, 512."""
        t = ctypes.c_int32(0)
        ms = (ctypes.c_double * 3)()
        self._check(load().lbm_batch_tuning(self.h, ctypes.byref(t), ms))
        return {"tile": t.value,
                "ms_per_step": dict(zip((128, 256, 512), list(ms)))}

    def set_tile(self, tile: int):
        self._check(load().lbm_batch_set_tile(self.h, int(tile)))

    def close(self):
        if getattr(self, "h", None):
            load().lbm_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _prim4(s):
    """(rho, u, p) or (rho, u, v, p) as four floats."""
    s = tuple(float(v) for v in s)
    return s if len(s) == 4 else (s[0], s[1], 0.0, s[2])


def make_grid2d(cfg, inner, outer, geom=PLANAR_X, a0=0.5, a1=0.5,
                radius=0.0, nsteps=0) -> lbm_grid2d:
    """One grid of a Batch2D: its configuration (2-D, F32), its initial
    state as Solver.init_riemann takes it, and its step count."""
    return lbm_grid2d(cfg, lbm_prim(*_prim4(inner)), lbm_prim(*_prim4(outer)),
                      geom, 0, a0, a1, radius, nsteps)


class Batch2D:
    """Many independent small 2-D grids advanced together (lbm_batch2d_*):
    two launches per lattice step for the whole batch."""

    def __init__(self, grids, stream=None):
        lib = load()
        arr = (lbm_grid2d * len(grids))(*grids)
        self.n = [g.cfg.nx * g.cfg.ny for g in grids]
        h = _H()
        st = lib.lbm_batch2d_create(arr, len(grids), stream, ctypes.byref(h))
        if st != OK:
            raise LbmError(st, "lbm_batch2d_create")
        self.h = h

    def _check(self, st):
        if st != OK:
            msg = load().lbm_batch2d_last_error(self.h)
            raise LbmError(st, msg.decode() if msg else "")

    def run(self, max_steps=-1):
        self._check(load().lbm_batch2d_run(self.h, int(max_steps)))

    def steps(self) -> int:
        s = ctypes.c_int64(0)
        self._check(load().lbm_batch2d_steps(self.h, ctypes.byref(s)))
        return s.value

    def moments(self, j) -> dict:
        n = self.n[j]
        out = {k: np.empty(n) for k in ("rho", "mx", "my", "rhoE", "p")}
        self._check(load().lbm_batch2d_moments(
            self.h, j, _dp(out["rho"]), _dp(out["mx"]), _dp(out["my"]),
            _dp(out["rhoE"]), _dp(out["p"]), n))
        return out

    def close(self):
        if getattr(self, "h", None):
            load().lbm_batch2d_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Pool:
    """Tube pool for continuous batching (lbm_pool_*)."""

    def __init__(self, capacity_nodes, max_slots=4096, precision=F32,
                 gamma=1.4, theta=0.5, kahan=1, stream=None):
        lib = load()
        h = _H()
        st = lib.lbm_pool_create(precision, gamma, theta, kahan,
                                 int(capacity_nodes), int(max_slots), stream,
                                 ctypes.byref(h))
        if st != OK:
            raise LbmError(st, "lbm_pool_create")
        self.h = h
        self.n = {}

    def _check(self, st):
        if st != OK:
            msg = load().lbm_pool_last_error(self.h)
            raise LbmError(st, msg.decode() if msg else "")

    def add(self, tube: lbm_tube) -> int:
        s = ctypes.c_int32(-1)
        self._check(load().lbm_pool_add(self.h, ctypes.byref(tube),
                                        ctypes.byref(s)))
        self.n[s.value] = tube.n
        return s.value

    def step(self):
        self._check(load().lbm_pool_step(self.h))

    def run(self, nsteps: int):
        """nsteps pool steps in one call."""
        self._check(load().lbm_pool_run(self.h, int(nsteps)))

    def progress(self, slot):
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(load().lbm_pool_progress(self.h, slot, ctypes.byref(a),
                                             ctypes.byref(b)))
        return a.value, b.value

    def read(self, slot) -> dict:
        n = self.n[slot]
        out = {k: np.empty(n) for k in ("rho", "mx", "rhoE", "p")}
        self._check(load().lbm_pool_read(self.h, slot, _dp(out["rho"]),
                                         _dp(out["mx"]), _dp(out["rhoE"]),
                                         _dp(out["p"]), n))
        return out

    def remove(self, slot):
        self._check(load().lbm_pool_remove(self.h, slot))
        self.n.pop(slot, None)

    def close(self):
        if getattr(self, "h", None):
            load().lbm_pool_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
