"""GPU parity of the relaxation-time step (tau != 1, eqs 4-5, per-packet
state) through the C ABI, against the FP64 oracle.

FP64: the collision and the gather round every operation on its own, in the
oracle's order (slots in table order for the moments, sources ascending then
corners for every slot's arrivals), so packets and moments must agree bit
for bit.  FP32: mean |error| at most 1e-5 of each field's range after a few
steps (the square lattice amplifies round-off; see the tau = 1 tests).
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

from paper_1602_02675_gb300 import lbm as L  # noqa: E402

T, R, P = L.TRANSMISSIVE, L.REFLECTING, L.PERIODIC


def _cfg(dim, nx, ny, bcx, bcy, precision, max_reach=0):
    return L.make_config(dim, nx, ny, dt=1.0 / nx, precision=precision,
                         bc_x=bcx, bc_y=bcy, max_reach=max_reach)


def _params(dim, nx, ny, bcx, bcy):
    return O.Params(dim=dim, nx=nx, ny=ny if dim == 2 else 1, bc_x=bcx,
                    bc_y=bcy)


def random_packets(dim, n, seed, spread=0.6):
    """Seeded non-equilibrium packets (slots, fields, nodes) with positive
    masses and internal energies: per slot a mass d, a velocity xi scattered
    about the slot's c' (level speeds 1 and 2), an internal part eps >= 0;
    stored as (d, d xi, d (|xi|^2/2 + eps))."""
    rng = np.random.default_rng(seed)
    if dim == 1:
        cs = [(0,), (1,), (-1,), (2,), (-2,)]
    else:
        cs = [(1, 0), (-1, 0), (0, 1), (0, -1), (2, 0), (-2, 0), (0, 2),
              (0, -2)]
    f = np.zeros((len(cs), dim + 2, n))
    for j, c in enumerate(cs):
        d = rng.uniform(0.02, 0.15, n)
        xi = [0.5 * c[a] + rng.uniform(-spread, spread, n) for a in range(dim)]
        eps = rng.uniform(0.0, 0.3, n)
        f[j, 0] = d
        for a in range(dim):
            f[j, 1 + a] = d * xi[a]
        f[j, dim + 1] = d * (0.5 * sum(x * x for x in xi) + eps)
    return f


def _assert_bitwise(a, b):
    assert a.shape == b.shape
    same = np.asarray(a).view(np.uint64) == np.asarray(b).view(np.uint64)
    if not np.all(same):
        bad = np.argwhere(~same)[0]
        raise AssertionError(f"first mismatch at {tuple(bad)}: "
                             f"{a[tuple(bad)]!r} vs {b[tuple(bad)]!r}")


def _l1(g, o):
    rng = np.max(o) - np.min(o)
    scale = rng if rng > 0 else max(np.max(np.abs(o)), 1e-300)
    return np.mean(np.abs(g - o)) / scale


CASES_2D = [
    ((P, P), (37, 29), 0.7), ((P, P), (37, 29), 1.6),
    ((T, R), (41, 19), 3.0), ((R, R), (33, 17), 1.25),
    ((R, P), (35, 9), 2.0), ((T, T), (30, 26), 1.6),
]


# max_reach 6: collision and gather kernels; 4: the one-launch step
@pytest.mark.parametrize("max_reach", [6, 4])
@pytest.mark.parametrize("bcs,shape,tau", CASES_2D)
def test_bgk_2d_fp64_bitwise(bcs, shape, tau, max_reach):
    nx, ny = shape
    f0 = random_packets(2, nx * ny, seed=nx * 101 + ny + bcs[0])
    steps = 6
    with L.Bgk(_cfg(2, nx, ny, *bcs, L.F64, max_reach=max_reach), tau) as g:
        g.set_packets(f0)
        g.step(steps)
        got = g.packets()
        gm = g.moments()
        diag = g.diagnostics()
    Pp = _params(2, nx, ny, *bcs)
    ref, ec = O.bgk_run(Pp, tau, f0, steps)
    _assert_bitwise(got, ref)
    om = O.bgk_moments(Pp, ref)
    for k, v in (("rho", om.rho), ("mx", om.mx), ("my", om.my),
                 ("rhoE", om.rhoE)):
        _assert_bitwise(gm[k], v)
    assert diag["eclamps"] == ec
    assert diag["flags"] == 0


@pytest.mark.parametrize("bc", [T, R, P])
@pytest.mark.parametrize("tau", [0.8, 1.5])
def test_bgk_1d_sod_fp64_bitwise(bc, tau):
    """Sod tube (Section V.C) from equilibrium; the initial packets come from
    the GPU's own init and equilibrium kernels."""
    n, steps = 400, 40
    with L.Bgk(_cfg(1, n, 1, bc, 0, L.F64), tau) as g:
        g.init_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), L.PLANAR_X, 0.5)
        f_init = g.packets()
        g.step(steps)
        got = g.packets()
    Pp = _params(1, n, 1, bc, 0)
    s = O.riemann_planar(Pp, 0.0, 1.0, 0.5, (1.0, 0.0, 1.0),
                         (0.125, 0.0, 0.1), 1.0)
    f0 = O.bgk_equilibrium(Pp, s)
    _assert_bitwise(f_init, f0)
    ref, _ = O.bgk_run(Pp, tau, f0, steps)
    _assert_bitwise(got, ref)


@pytest.mark.parametrize("bcs,shape,tau", CASES_2D[:4])
def test_bgk_2d_fp32_l1(bcs, shape, tau):
    nx, ny = shape
    f0 = random_packets(2, nx * ny, seed=nx * 103 + ny + bcs[1])
    steps = 4
    with L.Bgk(_cfg(2, nx, ny, *bcs, L.F32), tau) as g:
        g.set_packets(f0)
        g.step(steps)
        got = g.packets()
        gm = g.moments()
    Pp = _params(2, nx, ny, *bcs)
    f32_in = f0.astype(np.float32).astype(np.float64)
    ref, _ = O.bgk_run(Pp, tau, f32_in, steps)
    for c in range(4):
        assert _l1(got[:, c, :], ref[:, c, :]) <= 1e-5, c
    om = O.bgk_moments(Pp, ref)
    for k, v in (("rho", om.rho), ("mx", om.mx), ("my", om.my),
                 ("rhoE", om.rhoE)):
        assert _l1(gm[k], v) <= 1e-5, k


def test_bgk_1d_fp32_l1():
    n, steps, tau = 1000, 200, 1.5
    with L.Bgk(_cfg(1, n, 1, T, 0, L.F32), tau) as g:
        g.init_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), L.PLANAR_X, 0.5)
        g.step(steps)
        gm = g.moments()
    Pp = _params(1, n, 1, T, 0)
    s = O.riemann_planar(Pp, 0.0, 1.0, 0.5, (1.0, 0.0, 1.0),
                         (0.125, 0.0, 0.1), 1.0)
    ref, _ = O.bgk_run(Pp, tau, O.bgk_equilibrium(Pp, s), steps)
    om = O.bgk_moments(Pp, ref)
    for k, v in (("rho", om.rho), ("mx", om.mx), ("rhoE", om.rhoE)):
        assert _l1(gm[k], v) <= 1e-5, k


@pytest.mark.parametrize("prec", [L.F64, L.F32])
def test_bgk_tau_one_matches_the_moments_step(prec):
    """At tau = 1 the per-packet handle takes the same steps as the
    moments-only handle (eq 10): the same values up to the order of the
    sums, and within 1e-5 of the range in FP32."""
    nx, ny, steps = 48, 40, 10
    args = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), L.CIRCLE, 0.5,
            0.5, 0.3)
    with L.Bgk(_cfg(2, nx, ny, P, P, prec), 1.0) as g:
        g.init_riemann(*args)
        g.step(steps)
        gm = g.moments()
    with L.Solver(_cfg(2, nx, ny, P, P, prec)) as s:
        s.init_riemann(*args)
        s.step(steps)
        sm = s.moments()
    for k in ("rho", "mx", "my", "rhoE"):
        if prec == L.F64:
            assert np.max(np.abs(gm[k] - sm[k])) <= 1e-12 * np.max(np.abs(sm[k]))
        else:
            assert _l1(gm[k], sm[k]) <= 1e-5, k


# FP32: the packets are stored in FP32 after every step and the gather sums
# in plain FP32 (1.3e-6 of the mass and 2.8e-6 of the energy over these
# 100 steps on a GB300)
@pytest.mark.parametrize("prec,tol", [(L.F64, 1e-12), (L.F32, 1e-5)])
def test_bgk_conservation_periodic(prec, tol):
    nx, ny = 64, 48
    with L.Bgk(_cfg(2, nx, ny, P, P, prec), 1.7) as g:
        g.init_riemann((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1),
                       L.CIRCLE, 0.5, 0.5, 0.3)
        t0 = g.conservation()
        g.step(100)
        t1 = g.conservation()
    scale = max(abs(t0[0]), abs(t0[3]))
    assert np.all(np.abs(t1 - t0) <= tol * scale), (t1 - t0) / scale


@pytest.mark.parametrize("prec", [L.F64, L.F32])
def test_bgk_restart_is_bitwise(prec):
    """Packets read out and set into a fresh handle continue bit for bit."""
    nx, ny, tau = 40, 24, 1.4
    args = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), L.CIRCLE, 0.5,
            0.5, 0.3)
    with L.Bgk(_cfg(2, nx, ny, T, R, prec), tau) as g:
        g.init_riemann(*args)
        g.step(8)
        whole = g.packets()
    with L.Bgk(_cfg(2, nx, ny, T, R, prec), tau) as g:
        g.init_riemann(*args)
        g.step(3)
        mid = g.packets()
    with L.Bgk(_cfg(2, nx, ny, T, R, prec), tau) as g:
        g.set_packets(mid)
        g.step(5)
        _assert_bitwise(g.packets(), whole)


def test_bgk_errors_are_reported():
    nx = 32
    # a reach beyond max_reach: the state is left as it was
    f0 = random_packets(2, nx * nx, seed=9, spread=0.2)
    f0[:, 1, :] += 3.0 * f0[:, 0, :]          # V_x about 3
    with L.Bgk(_cfg(2, nx, nx, P, P, L.F64, max_reach=3), 1.5) as g:
        g.set_packets(f0)
        g.step(1)
        with pytest.raises(L.LbmError) as e:
            g.synchronize()
        assert e.value.status == L.EREACH
    with L.Bgk(_cfg(2, nx, nx, P, P, L.F64, max_reach=3), 1.5) as g:
        g.set_packets(f0)
        g.step(1)
        d = g.diagnostics()
        assert d["flags"] & 2
    # negative density
    f1 = random_packets(2, nx * nx, seed=10)
    f1[:, 0, 77] = -1.0
    with L.Bgk(_cfg(2, nx, nx, P, P, L.F32), 1.5) as g:
        g.set_packets(f1)
        g.step(1)
        with pytest.raises(L.LbmError) as e:
            g.synchronize()
        assert e.value.status == L.ESTATE
    with pytest.raises(L.LbmError):
        L.Bgk(_cfg(2, nx, nx, P, P, L.F32), 0.5)


def test_bgk_empty_nodes_emit_nothing():
    """Nodes whose slot masses sum to zero hold no packets and send none."""
    nx, ny, tau = 24, 16, 1.8
    f0 = random_packets(2, nx * ny, seed=11)
    f0[:, :, 5 * nx + 3: 5 * nx + 9] = 0.0
    f0[:, :, 11 * nx:12 * nx] = 0.0
    with L.Bgk(_cfg(2, nx, ny, P, R, L.F64), tau) as g:
        g.set_packets(f0)
        g.step(3)
        got = g.packets()
    ref, _ = O.bgk_run(_params(2, nx, ny, P, R), tau, f0, 3)
    _assert_bitwise(got, ref)


def test_bgk_benchmark_workload_sampled_fp32():
    """The benchmark's workload and launch configuration (2048^2 periodic
    cylinder, FP32, tau = 1.5, bench.py --workload bgk2d): after 20 steps,
    step 21 compared at sampled nodes with one oracle step of the patch of
    half-width max_reach around each (a node's new slots depend only on the
    sources within the step's reach, so the patch's own edges do not reach
    its centre)."""
    n, tau, H = 2048, 1.5, 4
    cfg = L.make_config(2, n, n, dt=1.0 / n, precision=L.F32, bc_x=P, bc_y=P,
                        max_reach=4)
    with L.Bgk(cfg, tau) as g:
        g.init_riemann((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1),
                       L.CIRCLE, 0.5, 0.5, 0.4)
        g.step(20)
        fk = g.packets()
        g.step(1)
        d = g.diagnostics()
        fk1 = g.packets()
    assert d["flags"] == 0 and d["reach"] <= H
    rng = np.random.default_rng(21)
    pts = [(int(x), int(y)) for x, y in rng.integers(0, n, (8, 2))]
    for ang in np.linspace(0.0, 2 * np.pi, 17)[:-1]:
        # on the circle's edge, where the flow is
        pts.append((int(n * (0.5 + 0.4 * np.cos(ang))) % n,
                    int(n * (0.5 + 0.4 * np.sin(ang))) % n))
    w = 2 * H + 1
    Pp = O.Params(dim=2, nx=w, ny=w, bc_x=O.TRANSMISSIVE,
                  bc_y=O.TRANSMISSIVE)
    for x, y in pts:
        xs = np.arange(x - H, x + H + 1) % n
        ys = np.arange(y - H, y + H + 1) % n
        idx = (ys[:, None] * n + xs[None, :]).ravel()
        out, _, _ = O.bgk_step(Pp, tau, fk[:, :, idx])
        o = out[:, :, H * w + H]
        gv = fk1[:, :, y * n + x]
        scale = np.max(np.abs(o), axis=0)
        assert np.all(np.abs(gv - o) <= 1e-5 * scale + 1e-30), (x, y)


@pytest.mark.parametrize("bcs,shape", [((P, P), (37, 29)), ((T, R), (130, 70)),
                                       ((R, P), (67, 41))])
def test_bgk_one_launch_equals_two_kernels_fp32(bcs, shape):
    """The one-launch step (max_reach <= 4) collides each tile's window in
    shared memory with the same arithmetic as the collision kernel and
    gathers in the same order: FP32 results identical bit for bit."""
    nx, ny = shape
    f0 = random_packets(2, nx * ny, seed=nx + 7 * ny)
    out = []
    for mr in (6, 4):
        with L.Bgk(_cfg(2, nx, ny, *bcs, L.F32, max_reach=mr), 1.6) as g:
            g.set_packets(f0)
            g.step(7)
            out.append((g.packets(), g.diagnostics()))
    _assert_bitwise(out[0][0], out[1][0])
    assert out[0][1]["reach"] == out[1][1]["reach"]
    assert out[0][1]["eclamps"] == out[1][1]["eclamps"]


def test_bgk_one_launch_cylinder_equals_two_kernels_fp32():
    n = 256
    args = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), L.CIRCLE, 0.5,
            0.5, 0.4)
    out = []
    for mr in (6, 4):
        cfg = L.make_config(2, n, n, dt=1.0 / n, precision=L.F32, bc_x=P,
                            bc_y=P, max_reach=mr)
        with L.Bgk(cfg, 1.5) as g:
            g.init_riemann(*args)
            g.step(60)
            out.append(g.packets())
    _assert_bitwise(out[0], out[1])


def test_bgk_one_launch_reach_limit():
    """A reach beyond 4 on the one-launch path: LBM_EREACH, and the packets
    are left as they were."""
    nx = 40
    f0 = random_packets(2, nx * nx, seed=12, spread=0.2)
    f0[:, 1, :] += 3.0 * f0[:, 0, :]          # V_x about 3: reach 5 or more
    with L.Bgk(_cfg(2, nx, nx, P, P, L.F64, max_reach=4), 1.5) as g:
        g.set_packets(f0)
        g.step(1)
        d = g.diagnostics()
        assert d["flags"] & 2
        with pytest.raises(L.LbmError) as e:
            g.synchronize()
        assert e.value.status == L.EREACH


def test_bgk_one_launch_restart_is_bitwise():
    nx, ny, tau = 40, 24, 1.4
    args = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), L.CIRCLE, 0.5,
            0.5, 0.3)
    cfg = lambda: _cfg(2, nx, ny, T, R, L.F32, max_reach=4)
    with L.Bgk(cfg(), tau) as g:
        g.init_riemann(*args)
        g.step(8)
        whole = g.packets()
    with L.Bgk(cfg(), tau) as g:
        g.init_riemann(*args)
        g.step(3)
        mid = g.packets()
    with L.Bgk(cfg(), tau) as g:
        g.set_packets(mid)
        g.step(5)
        _assert_bitwise(g.packets(), whole)


def test_bgk_one_launch_fp64_bitwise_many_tiles():
    """The one-launch step on a grid of 161 tiles with ragged right and
    bottom rows of tiles, reflecting walls in y: the oracle's bits."""
    nx, ny, tau, steps = 200, 184, 1.6, 4
    cfg = _cfg(2, nx, ny, P, R, L.F64, max_reach=4)
    args = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), L.CIRCLE, 0.5,
            0.45, 0.3)
    with L.Bgk(cfg, tau) as g:
        g.init_riemann(*args)
        f0 = g.packets()
        g.step(steps)
        got = g.packets()
        d = g.diagnostics()
    ref, ec = O.bgk_run(_params(2, nx, ny, P, R), tau, f0, steps)
    _assert_bitwise(got, ref)
    assert d["eclamps"] == ec and d["flags"] == 0


def test_bgk_one_launch_fp32_equals_two_kernels_many_tiles():
    """416 x 600 (975 tiles), 40 steps of the cylinder: FP32 identical bit
    for bit to the two-kernel step."""
    nx, ny = 416, 600
    args = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), L.CIRCLE, 0.5,
            0.7, 0.3)
    out = []
    for mr in (6, 4):
        with L.Bgk(_cfg(2, nx, ny, P, P, L.F32, max_reach=mr), 1.5) as g:
            g.init_riemann(*args)
            g.step(40)
            out.append((g.packets(), g.diagnostics()))
    _assert_bitwise(out[0][0], out[1][0])
    assert out[0][1]["reach"] == out[1][1]["reach"]
