"""Python face of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``liboracle.so`` built from
``lbm_oracle.c`` (plain C, FP64, ``-ffp-contract=off``) and adds the parts of
the method that sit outside the step:

* physical <-> lattice units (lattice velocity V = u*lambda, energies per unit
  mass scale with lambda^2, lambda = dt/dx);
* the Sod / cylindrical Riemann initial states of Section V.C;
* pressure recovery P = (gamma-1) rho e (eq 27);
* the per-packet state of the relaxation-time step (tau != 1, eqs 4-5):
  equilibrium packets of given moments, moments of packets, steps.

It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TRANSMISSIVE, REFLECTING, PERIODIC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, FP64, no contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("bc_x", ctypes.c_int32),
                ("bc_y", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("gamma", ctypes.c_double), ("theta", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        pp = ctypes.POINTER(_Params)
        lib.ora_step.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, i64p, i64p]
        lib.ora_run.argtypes = [pp, dp, dp, dp, dp, ctypes.c_int64, i64p]
        lib.ora_reach.argtypes = [pp, dp, dp, dp, dp, i64p]
        lib.ora_equilibrium_probe.argtypes = [pp, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, dp]
        lib.ora_packets_probe.argtypes = [pp, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp]
        lib.ora_bgk_equilibrium.argtypes = [pp, dp, dp, dp, dp, dp]
        lib.ora_bgk_moments.argtypes = [pp, dp, dp, dp, dp, dp]
        lib.ora_bgk_step.argtypes = [pp, ctypes.c_double, dp, dp, i64p, i64p]
        lib.ora_bgk_run.argtypes = [pp, ctypes.c_double, dp, ctypes.c_int64,
                                    i64p]
        for f in (lib.ora_step, lib.ora_run, lib.ora_reach,
                  lib.ora_equilibrium_probe, lib.ora_packets_probe,
                  lib.ora_bgk_equilibrium, lib.ora_bgk_moments,
                  lib.ora_bgk_step, lib.ora_bgk_run):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Params:
    """Lattice and gas of one run (Sections III-V)."""
    dim: int
    nx: int
    ny: int = 1
    gamma: float = 1.4
    theta: float = 0.5
    bc_x: int = TRANSMISSIVE
    bc_y: int = REFLECTING

    def c(self) -> _Params:
        return _Params(self.dim, self.bc_x, self.bc_y, 0, self.nx,
                       self.ny if self.dim == 2 else 1, self.gamma, self.theta)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


@dataclass
class State:
    """Lattice-unit moments of every node (x fastest).  my is None in 1-D."""
    rho: np.ndarray
    mx: np.ndarray
    my: np.ndarray | None
    rhoE: np.ndarray

    def copy(self) -> "State":
        return State(self.rho.copy(), self.mx.copy(),
                     None if self.my is None else self.my.copy(),
                     self.rhoE.copy())

    def fields(self):
        return [f for f in (self.rho, self.mx, self.my, self.rhoE)
                if f is not None]


def _arrays(P: Params, s: State):
    out = []
    for f in (s.rho, s.mx, s.my if P.dim == 2 else s.rho, s.rhoE):
        out.append(np.ascontiguousarray(f, dtype=np.float64))
    return out


def step(P: Params, s: State) -> tuple[State, int, int]:
    """One tau = 1 step.  Returns (new state, e-clamp count, reach used)."""
    lib = _load()
    r, x, y, e = _arrays(P, s)
    n = P.nx * (P.ny if P.dim == 2 else 1)
    ro, xo, eo = (np.empty(n) for _ in range(3))
    yo = np.empty(n) if P.dim == 2 else None
    ec, R = ctypes.c_int64(0), ctypes.c_int64(0)
    p = P.c()
    st = lib.ora_step(ctypes.byref(p), _dp(r), _dp(x), _dp(y), _dp(e),
                      _dp(ro), _dp(xo), _dp(yo) if yo is not None else None,
                      _dp(eo), ctypes.byref(ec), ctypes.byref(R))
    if st != 0:
        raise OracleError(f"ora_step status {st}")
    return State(ro, xo, yo, eo), ec.value, R.value


def run(P: Params, s: State, nsteps: int) -> tuple[State, int]:
    """nsteps steps; returns (state, total e-clamp count)."""
    lib = _load()
    r, x, y, e = (a.copy() for a in _arrays(P, s))
    ec = ctypes.c_int64(0)
    p = P.c()
    st = lib.ora_run(ctypes.byref(p), _dp(r), _dp(x),
                     _dp(y) if P.dim == 2 else None, _dp(e), nsteps,
                     ctypes.byref(ec))
    if st != 0:
        raise OracleError(f"ora_run status {st}")
    return State(r, x, y if P.dim == 2 else None, e), ec.value


def reach(P: Params, s: State) -> int:
    lib = _load()
    r, x, y, e = _arrays(P, s)
    R = ctypes.c_int64(0)
    p = P.c()
    st = lib.ora_reach(ctypes.byref(p), _dp(r), _dp(x), _dp(y), _dp(e),
                       ctypes.byref(R))
    if st != 0:
        raise OracleError(f"ora_reach status {st}")
    return R.value


def equilibrium(P: Params, rho, mx, my, rhoE) -> dict:
    """Equilibrium quantities of one lattice-unit state (eqs 13-15, 24-26)."""
    lib = _load()
    out = np.zeros(11)
    p = P.c()
    st = lib.ora_equilibrium_probe(ctypes.byref(p), rho, mx, my, rhoE,
                                   _dp(out))
    if st != 0:
        raise OracleError(f"ora_equilibrium status {st}")
    keys = ("c1", "c2", "d0", "d1", "d2", "phi", "e", "nx", "fx", "ny", "fy")
    return dict(zip(keys, out.tolist()))


def packets(P: Params, rho, mx, my, rhoE) -> np.ndarray:
    """Rows (c'_x, c'_y, mass, mom_x, mom_y, energy) of one state's packets."""
    lib = _load()
    out = np.zeros(48)
    p = P.c()
    n = lib.ora_packets_probe(ctypes.byref(p), rho, mx, my, rhoE, _dp(out))
    return out[:6 * n].reshape(n, 6)


# ----------------------------------------------------------------------------
# relaxation time tau != 1 (eqs 4-5): per-packet state
# ----------------------------------------------------------------------------

def slots(dim: int) -> int:
    """Packet slots per node: the velocity set's entries (Section IV)."""
    return 5 if dim == 1 else 8


def packet_fields(dim: int) -> int:
    """Fields per slot: mass, momentum per axis, energy."""
    return dim + 2


def bgk_equilibrium(P: Params, s: State) -> np.ndarray:
    """Per-packet state at equilibrium with the moments s, shaped
    (slots, fields, nodes)."""
    lib = _load()
    r, x, y, e = _arrays(P, s)
    n = r.size
    f = np.zeros((slots(P.dim), packet_fields(P.dim), n))
    p = P.c()
    st = lib.ora_bgk_equilibrium(ctypes.byref(p), _dp(r), _dp(x),
                                 _dp(y) if P.dim == 2 else None, _dp(e),
                                 _dp(f))
    if st != 0:
        raise OracleError(f"ora_bgk_equilibrium status {st}")
    return f


def bgk_moments(P: Params, f: np.ndarray) -> State:
    """Moments of every node, the sum of its slots (eq 6)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.shape[-1]
    r, x, e = (np.empty(n) for _ in range(3))
    y = np.empty(n) if P.dim == 2 else None
    p = P.c()
    st = lib.ora_bgk_moments(ctypes.byref(p), _dp(f), _dp(r), _dp(x),
                             _dp(y) if y is not None else None, _dp(e))
    if st != 0:
        raise OracleError(f"ora_bgk_moments status {st}")
    return State(r, x, y, e)


def bgk_step(P: Params, tau: float, f: np.ndarray):
    """One step with relaxation time tau.  Returns (new f, e-clamp count,
    reach used)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    ec, R = ctypes.c_int64(0), ctypes.c_int64(0)
    p = P.c()
    st = lib.ora_bgk_step(ctypes.byref(p), float(tau), _dp(f), _dp(out),
                          ctypes.byref(ec), ctypes.byref(R))
    if st != 0:
        raise OracleError(f"ora_bgk_step status {st}")
    return out, ec.value, R.value


def bgk_run(P: Params, tau: float, f: np.ndarray, nsteps: int):
    """nsteps steps with relaxation time tau; returns (f, e-clamp count)."""
    lib = _load()
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    ec = ctypes.c_int64(0)
    p = P.c()
    st = lib.ora_bgk_run(ctypes.byref(p), float(tau), _dp(f), int(nsteps),
                         ctypes.byref(ec))
    if st != 0:
        raise OracleError(f"ora_bgk_run status {st}")
    return f, ec.value


# ----------------------------------------------------------------------------
# units and initial states (Section V.C)
# ----------------------------------------------------------------------------

def steps_and_lambda(t_end: float, dx: float) -> tuple[int, float]:
    """Number of steps with lambda = dt/dx close to 1 that lands on t_end
    exactly: n = ceil(t_end/dx - 1e-9), lambda = t_end/(n dx)."""
    n = int(math.ceil(t_end / dx - 1e-9))
    n = max(n, 1)
    return n, t_end / (n * dx)


def prims_to_lattice(gamma: float, lam: float, rho, u, v, p) -> State:
    """Physical primitives -> lattice-unit moments:
    m = rho u lambda, rhoE = p lambda^2/(gamma-1) + rho |u lambda|^2 / 2."""
    rho = np.asarray(rho, dtype=np.float64)
    Vx = np.asarray(u, dtype=np.float64) * lam
    Vy = None if v is None else np.asarray(v, dtype=np.float64) * lam
    p = np.asarray(p, dtype=np.float64)
    kin = Vx * Vx if Vy is None else Vx * Vx + Vy * Vy
    rhoE = p * lam * lam / (gamma - 1.0) + 0.5 * rho * kin
    return State(rho.copy(), rho * Vx, None if Vy is None else rho * Vy, rhoE)


def lattice_to_physical(gamma: float, lam: float, s: State) -> dict:
    """Lattice moments -> physical conserved fields and pressure (eq 27)."""
    rho = s.rho
    mx = s.mx / lam
    my = None if s.my is None else s.my / lam
    rhoE = s.rhoE / (lam * lam)
    kin = mx * mx if my is None else mx * mx + my * my
    with np.errstate(divide="ignore", invalid="ignore"):
        p = (gamma - 1.0) * (rhoE - 0.5 * kin / rho)
        u = mx / rho
        v = None if my is None else my / rho
    return dict(rho=rho, mx=mx, my=my, rhoE=rhoE, p=p, u=u, v=v)


def node_x(nx: int, x0: float, x1: float) -> np.ndarray:
    """Cell-centred node positions x_i = x0 + (i + 1/2) dx."""
    dx = (x1 - x0) / nx
    return x0 + (np.arange(nx) + 0.5) * dx


def riemann_planar(P: Params, x0: float, x1: float, x_d: float, left, right,
                   lam: float) -> State:
    """Planar jump along x at x_d: nodes with x < x_d take `left`, the rest
    `right`.  left/right are (rho, u, p) or (rho, u, v, p)."""
    x = node_x(P.nx, x0, x1)
    ny = P.ny if P.dim == 2 else 1
    X = np.tile(x, ny)
    inside = X < x_d
    return _assign(P, inside, left, right, lam)


def riemann_circle(P: Params, x0: float, x1: float, y0: float, cx: float,
                   cy: float, radius: float, inner, outer,
                   lam: float) -> State:
    """Circle: nodes with (x-cx)^2 + (y-cy)^2 < radius^2 take `inner`."""
    dx = (x1 - x0) / P.nx
    x = node_x(P.nx, x0, x1)
    y = y0 + (np.arange(P.ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    r2 = (X - cx) * (X - cx) + (Y - cy) * (Y - cy)
    inside = (r2 < radius * radius).ravel()
    return _assign(P, inside, inner, outer, lam)


def _prim4(s):
    s = tuple(float(v) for v in s)
    return s if len(s) == 4 else (s[0], s[1], 0.0, s[2])


def _assign(P: Params, inside: np.ndarray, a, b, lam: float) -> State:
    a, b = _prim4(a), _prim4(b)
    pick = lambda i: np.where(inside, a[i], b[i])
    rho, u, v, p = (pick(i) for i in range(4))
    return prims_to_lattice(P.gamma, lam, rho, u, v if P.dim == 2 else None, p)


def totals(s: State) -> np.ndarray:
    """Plain sums of the lattice moments over all nodes (FP64)."""
    my = 0.0 if s.my is None else float(np.sum(s.my))
    return np.array([np.sum(s.rho), np.sum(s.mx), my, np.sum(s.rhoE)])
