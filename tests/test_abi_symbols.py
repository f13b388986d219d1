"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/lbm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(lbm_\w+)\s*\(", text,
                             flags=re.M):
            if not m.group(0).lstrip().startswith("typedef"):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_02675_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_core_entry_points():
    names = _declared()
    for core in ("lbm_create", "lbm_init_riemann", "lbm_step", "lbm_moments",
                 "lbm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version_and_null_safety(lib):
    lib.lbm_abi_version.restype = ctypes.c_int32
    assert lib.lbm_abi_version() >= 1
    lib.lbm_destroy.argtypes = [ctypes.c_void_p]
    lib.lbm_destroy(None)            # NULL-safe, no CUDA call
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_last_error.argtypes = [ctypes.c_void_p]
    assert lib.lbm_last_error(None)
    lib.lbm_lambda.restype = ctypes.c_double
    lib.lbm_lambda.argtypes = [ctypes.c_void_p]
    assert lib.lbm_lambda(None) == 0.0


def test_binding_names_match_the_abi():
    from paper_1602_02675_gb300 import lbm as L
    lib = L.load()
    for n in _declared():
        assert getattr(lib, n).argtypes is not None or n == "lbm_abi_version"


def test_bgk_create_checks_tau_before_any_cuda_call():
    """tau must be finite and above 1/2 (eqs 4-5); the check comes before
    any allocation, so it runs here without a GPU."""
    from paper_1602_02675_gb300 import lbm as L
    lib = L.load()
    cfg = L.make_config(1, 64, bc_x=L.PERIODIC)
    h = ctypes.c_void_p()
    for tau in (0.5, 0.25, -1.0, float("nan"), float("inf")):
        assert lib.lbm_bgk_create(ctypes.byref(cfg), tau,
                                  ctypes.byref(h)) == L.EINVAL
        assert not h.value
    lib.lbm_bgk_destroy(None)
    assert lib.lbm_bgk_last_error(None)


def test_bgk_create_checks_the_grid_before_any_cuda_call():
    from paper_1602_02675_gb300 import lbm as L
    lib = L.load()
    h = ctypes.c_void_p()
    bad = [L.make_config(2, 64, 8 * 65535 + 1, bc_x=L.PERIODIC),  # launch rows
           L.make_config(1, 16, bc_x=L.PERIODIC, dt=-1.0),          # dt <= 0
           L.make_config(2, 64, 64, theta=0.5)]                     # 2-D theta
    for cfg in bad:
        assert lib.lbm_bgk_create(ctypes.byref(cfg), 1.5,
                                  ctypes.byref(h)) == L.EINVAL
        assert not h.value


def test_create_calls_reject_the_same_bad_configs():
    """lbm_create and lbm_bgk_create share one configuration check; every
    rejection happens before any CUDA call, so it runs here without a GPU."""
    from paper_1602_02675_gb300 import lbm as L
    lib = L.load()
    mk = L.make_config
    bad = [mk(3, 16),                                       # dim
           mk(1, 16, precision=7),                          # precision
           mk(2, 16, 0),                                    # ny < 1
           mk(1, 16, bc_x=5),                               # boundary kind
           mk(2, 16, 16, bc_y=-1),
           mk(1, 16, gamma=1.0),                            # gamma <= 1
           mk(1, 16, x0=1.0, x1=0.5),                       # extent
           mk(1, 16, dt=0.0),                               # dt
           mk(1, 16, theta=1.0),                            # 1-D theta
           mk(2, 16, 16, theta=0.5),                        # 2-D theta
           mk(1, 16, max_reach=-1),
           mk(2, 1 << 20, 1 << 12)]                         # nx ny > 2^31 - 1
    for cfg in bad:
        h = ctypes.c_void_p()
        assert lib.lbm_create(ctypes.byref(cfg), ctypes.byref(h)) == L.EINVAL
        assert not h.value
        assert lib.lbm_bgk_create(ctypes.byref(cfg), 1.5,
                                  ctypes.byref(h)) == L.EINVAL
        assert not h.value


def test_create_calls_accept_valid_configs():
    """Valid configurations pass the shared check: without a GPU the call
    then fails in CUDA (not LBM_EINVAL); with one it makes a handle."""
    from paper_1602_02675_gb300 import lbm as L
    lib = L.load()
    good = [L.make_config(1, 1000, bc_x=L.TRANSMISSIVE),
            L.make_config(2, 64, 48, precision=L.F32, bc_x=L.PERIODIC,
                          bc_y=L.PERIODIC, max_reach=4),
            L.make_config(2, 40, 24, bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING)]
    for cfg in good:
        h = ctypes.c_void_p()
        st = lib.lbm_create(ctypes.byref(cfg), ctypes.byref(h))
        assert st != L.EINVAL
        if st == L.OK:
            lib.lbm_destroy(h)
        st = lib.lbm_bgk_create(ctypes.byref(cfg), 1.5, ctypes.byref(h))
        assert st != L.EINVAL
        if st == L.OK:
            lib.lbm_bgk_destroy(h)
