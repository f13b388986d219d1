"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64: the step sums every destination's arrivals in the same order as the
oracle and rounds each product and sum on its own, so the results must be
identical bit for bit (the 1e-12 relative bar is implied).  FP32: mean
absolute error at most 1e-5 of each field's range.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1602_02675_gb300 import inputs as I

pytestmark = pytest.mark.gpu

from paper_1602_02675_gb300 import lbm as L  # noqa: E402

FIELDS = ("rho", "mx", "my", "rhoE")


def _gpu(dim, nx, ny, bc_x, bc_y, prims=None, riemann=None, steps=1,
         precision=None, lam=1.0, kahan=1, max_reach=0):
    precision = L.F64 if precision is None else precision
    dx = 1.0 / nx
    cfg = L.make_config(dim, nx, ny, dt=lam * dx, precision=precision,
                        bc_x=bc_x, bc_y=bc_y, kahan=kahan, max_reach=max_reach)
    with L.Solver(cfg) as s:
        if prims is not None:
            s.set_primitives(*prims)
        else:
            s.init_riemann(*riemann)
        s.step(steps)
        out = s.moments()
        out["reach"] = s.reach()
        out["diag"] = s.diagnostics()
    return out


def _oracle(dim, nx, ny, bc_x, bc_y, prims=None, riemann=None, steps=1,
            lam=1.0):
    P = O.Params(dim=dim, nx=nx, ny=ny if dim == 2 else 1, bc_x=bc_x,
                 bc_y=bc_y)
    if prims is not None:
        st = O.prims_to_lattice(1.4, lam, prims[0], prims[1], prims[2],
                                prims[3])
    else:
        inner, outer, geom, a0, a1, r = riemann
        if geom == 0:
            st = O.riemann_planar(P, 0.0, 1.0, a0, inner, outer, lam)
        else:
            st = O.riemann_circle(P, 0.0, 1.0, 0.0, a0, a1, r, inner, outer,
                                  lam)
    st2, ec = O.run(P, st, steps)
    ph = O.lattice_to_physical(1.4, lam, st2)
    ph["eclamps"] = ec
    ph["reach"] = O.reach(P, st2)
    return ph


def _assert_bitwise(g, o, dim):
    for f in FIELDS:
        if f == "my" and dim == 1:
            continue
        assert np.array_equal(g[f], o[f]), (
            f, np.max(np.abs(g[f] - o[f])), np.argmax(np.abs(g[f] - o[f])))
        # the same bits, signs of zeros included
        assert np.array_equal(np.asarray(g[f], np.float64).view(np.uint64),
                              np.asarray(o[f], np.float64).view(np.uint64)), f
    np.testing.assert_allclose(g["p"], o["p"], rtol=1e-12,
                               atol=1e-12 * np.max(np.abs(o["p"])))


def _assert_l1(g, o, dim, tol=1e-5):
    for f in FIELDS:
        if f == "my" and dim == 1:
            continue
        rng = np.max(o[f]) - np.min(o[f])
        scale = rng if rng > 0 else max(np.max(np.abs(o[f])), 1e-300)
        err = np.mean(np.abs(g[f] - o[f])) / scale
        assert err <= tol, (f, err)


SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0, 0.5, 0.5, 0.0)


def test_sod_1d_fp64_bitwise():
    """1-D Sod tube, 1000 nodes, 200 steps to t = 0.2 (lambda = 1)."""
    g = _gpu(1, 1000, 1, L.TRANSMISSIVE, 0, riemann=SOD, steps=200)
    o = _oracle(1, 1000, 1, O.TRANSMISSIVE, 0, riemann=SOD, steps=200)
    _assert_bitwise(g, o, 1)
    assert g["reach"] >= o["reach"]


@pytest.mark.parametrize("bc", [L.TRANSMISSIVE, L.REFLECTING, L.PERIODIC])
@pytest.mark.parametrize("n", [1, 7, 300, 777])
def test_random_1d_fp64_bitwise(bc, n):
    """Independent random node states (every level count, both velocity
    signs) over several tiles with a ragged tail and degenerate sizes."""
    prims = I.random_node_prims(1, n, seed=1000 + n + bc)
    g = _gpu(1, n, 1, bc, 0, prims=prims, steps=3)
    o = _oracle(1, n, 1, bc, 0, prims=prims, steps=3)
    _assert_bitwise(g, o, 1)
    assert g["diag"]["eclamps"] == o["eclamps"]


BC2 = [(L.TRANSMISSIVE, L.REFLECTING), (L.PERIODIC, L.PERIODIC),
       (L.REFLECTING, L.TRANSMISSIVE), (L.TRANSMISSIVE, L.PERIODIC)]


@pytest.mark.parametrize("bcs", BC2)
@pytest.mark.parametrize("shape", [(70, 21), (33, 9), (3, 2)])
def test_random_2d_fp64_bitwise(bcs, shape):
    nx, ny = shape
    prims = I.random_smooth_prims(2, nx, ny, seed=2000 + nx + 7 * ny + bcs[0])
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=4)
    o = _oracle(2, nx, ny, *bcs, prims=prims, steps=4)
    _assert_bitwise(g, o, 2)


@pytest.mark.parametrize("bcs", [(L.PERIODIC, L.PERIODIC),
                                 (L.TRANSMISSIVE, L.REFLECTING)])
@pytest.mark.parametrize("bands,p_over_rho", [
    (((0.1, 0.8), (-0.8, -0.1)), 1.0),   # c1 = 1, n = (0, -1)
    (((-0.8, -0.1), (0.1, 0.8)), 0.3),   # c1 = 0, n = (-1, 0)
    (((0.1, 0.8), (0.1, 0.8)), 3.0),     # c1 = 2, n = (0, 0)
    (((-0.8, -0.1), (-0.8, -0.1)), 1.0)])
def test_one_type_windows_fp64_bitwise(bcs, bands, p_over_rho):
    """Every node of the first state has the same level speeds and lattice
    shift, so the interior windows take the compile-time landings; the
    result must still match the oracle's scan order bit for bit."""
    nx, ny = 100, 44
    prims = I.banded_prims(nx, ny, seed=3100 + int(10 * p_over_rho),
                           u_band=bands[0], v_band=bands[1],
                           p_over_rho=p_over_rho)
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=3)
    o = _oracle(2, nx, ny, *bcs, prims=prims, steps=3)
    _assert_bitwise(g, o, 2)


@pytest.mark.parametrize("bcs", [(L.PERIODIC, L.PERIODIC),
                                 (L.TRANSMISSIVE, L.REFLECTING)])
@pytest.mark.parametrize("bands,p_over_rho", [
    (((1.1, 1.6), (-0.4, 0.4)), 3.0),    # n_x = 1, c1 = 2: reach 5
    (((-1.6, -1.1), (1.1, 1.6)), 1.0)])  # n_x = -2, n_y = 1
def test_fast_flow_parity(bcs, bands, p_over_rho):
    """Lattice velocities beyond one node per step (shifts outside the
    compile-time landing lists, reach up to 5 of the 6 the records and
    windows hold): FP64 bit for bit, the FP32 kernels within 1e-5 of
    range."""
    nx, ny = 60, 36
    prims = I.banded_prims(nx, ny, seed=3400, u_band=bands[0],
                           v_band=bands[1], p_over_rho=p_over_rho)
    o = _oracle(2, nx, ny, *bcs, prims=prims, steps=4)
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=4)
    _assert_bitwise(g, o, 2)
    for kahan in (0, 1):
        g = _gpu(2, nx, ny, *bcs, prims=prims, steps=4, precision=L.F32,
                 kahan=kahan)
        _assert_l1(g, o, 2)


@pytest.mark.parametrize("kahan", [0, 1])
@pytest.mark.parametrize("bcs", [(L.PERIODIC, L.PERIODIC),
                                 (L.TRANSMISSIVE, L.REFLECTING)])
def test_patchwork_windows_many_groups_fp32_l1(bcs, kahan):
    """Windows holding several level speeds and lattice shifts of both
    signs on both axes: the mixed-window kernel's group walks (blocks of 1
    to 3 shifts, several groups per tile, minima carried from step to
    step).  FP32 within 1e-5 of range of the oracle after 1 and 4 steps."""
    nx, ny = 150, 110
    prims = I.patch_prims(nx, ny, seed=13)
    for steps in (1, 4):
        o = _oracle(2, nx, ny, *bcs, prims=prims, steps=steps)
        g = _gpu(2, nx, ny, *bcs, prims=prims, steps=steps, precision=L.F32,
                 kahan=kahan)
        assert g["diag"]["flags"] == 0
        _assert_l1(g, o, 2)


@pytest.mark.parametrize("kahan", [0, 1])
@pytest.mark.parametrize("seed", [14, 15])
def test_fp32_square_step_depends_on_state_only(seed, kahan):
    """The deposit kernels keep per-tile records of the windows they met
    (starting guesses for the next step).  The result must not depend on
    them: steps taken after checkpoints into fresh handles, whose records
    are empty, equal the uninterrupted run bit for bit (lambda = 1, so the
    checkpoint is exact)."""
    nx, ny = 150, 110
    prims = I.patch_prims(nx, ny, seed=seed)
    cfg = L.make_config(2, nx, ny, precision=L.F32, bc_x=L.PERIODIC,
                        bc_y=L.PERIODIC, kahan=kahan)
    with L.Solver(cfg) as a:
        a.set_primitives(*prims)
        a.step(6)
        ref = a.moments()
    m = None
    for part in (2, 3, 1):
        with L.Solver(cfg) as b:
            if m is None:
                b.set_primitives(*prims)
            else:
                b.set_moments(m["rho"], m["mx"], m["my"], m["rhoE"])
            b.step(part)
            m = b.moments()
    for f in FIELDS:
        assert np.array_equal(m[f], ref[f]), f


def test_fp32_reach_limit_beyond_deposit_window():
    """max_reach 8 exceeds the deposit kernel's window (reach 6), so the
    FP32 handle steps with the exact-order kernel instead; same results
    within the FP32 bar, and FP64 with the same limit (records padded by 8)
    bit for bit."""
    nx, ny = 70, 40
    prims = I.random_smooth_prims(2, nx, ny, seed=3500)
    bcs = (L.PERIODIC, L.REFLECTING)
    o = _oracle(2, nx, ny, *bcs, prims=prims, steps=5)
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=5, precision=L.F32,
             kahan=0, max_reach=8)
    _assert_l1(g, o, 2)
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=5, max_reach=8)
    _assert_bitwise(g, o, 2)


def test_vacuum_nodes_2d():
    """Nodes with zero density emit nothing (they only receive): FP64 bit
    for bit with the oracle, FP32 kernels within 1e-5 of range."""
    nx, ny = 70, 33
    rho, u, v, p = I.random_smooth_prims(2, nx, ny, seed=3600, jump=False)
    rng = np.random.default_rng(3601)
    empty = rng.choice(nx * ny, 60, replace=False)
    rho = rho.copy()
    p = p.copy()
    rho[empty] = 0.0
    p[empty] = 0.0
    prims = (rho, u, v, p)
    bcs = (L.TRANSMISSIVE, L.REFLECTING)
    o = _oracle(2, nx, ny, *bcs, prims=prims, steps=3)
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=3)
    _assert_bitwise(g, o, 2)
    for kahan in (0, 1):
        g = _gpu(2, nx, ny, *bcs, prims=prims, steps=3, precision=L.F32,
                 kahan=kahan)
        _assert_l1(g, o, 2)


@pytest.mark.parametrize("max_reach", [0, 4])
def test_closed_box_fp64_bitwise(max_reach):
    """Reflecting walls on all four sides (mirror images at the corners),
    with the default reach limit and a smaller one (the FP64 source
    records are padded by the limit)."""
    nx, ny = 70, 37
    prims = I.banded_prims(nx, ny, seed=3300, u_band=(0.1, 0.8),
                           v_band=(-0.8, -0.1), p_over_rho=1.0)
    g = _gpu(2, nx, ny, L.REFLECTING, L.REFLECTING, prims=prims, steps=6,
             max_reach=max_reach)
    o = _oracle(2, nx, ny, O.REFLECTING, O.REFLECTING, prims=prims, steps=6)
    _assert_bitwise(g, o, 2)
    assert g["diag"]["flags"] == 0


def test_sod_2d_paper_lattice_fp64_bitwise():
    """The paper's 400 x 4 square lattice (Section V.C) with x-only data."""
    lam = 1.0
    g = _gpu(2, 400, 4, L.TRANSMISSIVE, L.PERIODIC, riemann=SOD, steps=80)
    o = _oracle(2, 400, 4, O.TRANSMISSIVE, O.PERIODIC, riemann=SOD, steps=80)
    _assert_bitwise(g, o, 2)
    r = g["rho"].reshape(4, 400)
    assert np.array_equal(r, np.broadcast_to(r[0], r.shape))


def test_cylinder_fp64_bitwise():
    riem = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 1, 0.5, 0.5, 0.4)
    g = _gpu(2, 64, 64, L.PERIODIC, L.PERIODIC, riemann=riem, steps=30)
    o = _oracle(2, 64, 64, O.PERIODIC, O.PERIODIC, riemann=riem, steps=30)
    _assert_bitwise(g, o, 2)


def _golden_hashes(name):
    import os
    out = {}
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            n, steps, f, h = line.split()
            out[f] = (int(n), int(steps), h)
    return out


def test_cylinder_2000_steps_fp64_bitwise():
    """The periodic cylinder over a whole 2000-step solve on a 128 x 128
    lattice: the FP64 step reproduces the oracle's final state bit for bit
    (SHA-256 of every field, stored by tests/golden/make_golden.py), although
    the square-lattice step amplifies any round-off difference to O(1)
    within a few hundred steps."""
    import hashlib
    want = _golden_hashes("cylinder128_fp64_2000_sha256.txt")
    n, steps, _ = want["rho"]
    riem = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 1, 0.5, 0.5, 0.4)
    g = _gpu(2, n, n, L.PERIODIC, L.PERIODIC, riemann=riem, steps=steps)
    for f in FIELDS:
        h = hashlib.sha256(np.ascontiguousarray(g[f], "<f8").tobytes())
        assert h.hexdigest() == want[f][2], f


@pytest.mark.parametrize("kahan", [0, 1])
def test_cylinder_fp32_early_steps_l1(kahan):
    """FP32 against the oracle on the periodic cylinder (64 x 64) while the
    oracle's own FP32-storage floor is below the bar (100 steps: ~7e-7,
    tests/golden/cylinder_fp32_storage_floor.txt)."""
    riem = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 1, 0.5, 0.5, 0.4)
    g = _gpu(2, 64, 64, L.PERIODIC, L.PERIODIC, riemann=riem, steps=100,
             precision=L.F32, kahan=kahan)
    o = _oracle(2, 64, 64, O.PERIODIC, O.PERIODIC, riemann=riem, steps=100)
    _assert_l1(g, o, 2)


def test_lambda_not_one_fp64_bitwise():
    """Section V.C tube on 4096 nodes: 820 steps, lambda = 0.99902..."""
    nx = 4096
    n, lam = O.steps_and_lambda(0.2, 1.0 / nx)
    g = _gpu(1, nx, 1, L.TRANSMISSIVE, 0, riemann=SOD, steps=n, lam=lam)
    o = _oracle(1, nx, 1, O.TRANSMISSIVE, 0, riemann=SOD, steps=n, lam=lam)
    _assert_bitwise(g, o, 1)


TORO1 = ((1.0, 0.75, 1.0), (0.125, 0.0, 0.1), 0, 0.3, 0.5, 0.0)


@pytest.mark.parametrize("riem", [SOD, TORO1])
def test_lambda_half_fp64_bitwise(riem):
    """lambda = 0.5 (the oracle's conversion is pinned there by the
    conservation laws and the exact Riemann solution): a 1-D tube with a
    moving left state, 160 steps, and the same jump on a 2-D lattice between
    reflecting walls, through the GPU's own unit conversions."""
    g = _gpu(1, 400, 1, L.TRANSMISSIVE, 0, riemann=riem, steps=160, lam=0.5)
    o = _oracle(1, 400, 1, O.TRANSMISSIVE, 0, riemann=riem, steps=160,
                lam=0.5)
    _assert_bitwise(g, o, 1)
    r2 = ((riem[0][0], riem[0][1], 0.0, riem[0][2]),
          (riem[1][0], riem[1][1], 0.0, riem[1][2])) + riem[2:]
    g = _gpu(2, 96, 6, L.TRANSMISSIVE, L.REFLECTING, riemann=r2, steps=40,
             lam=0.5)
    o = _oracle(2, 96, 6, O.TRANSMISSIVE, O.REFLECTING, riemann=r2, steps=40,
                lam=0.5)
    _assert_bitwise(g, o, 2)
    prims = I.random_smooth_prims(2, 40, 24, seed=77)
    for prec, kahan in ((L.F32, 0), (L.F32, 1)):
        g = _gpu(2, 40, 24, L.PERIODIC, L.PERIODIC, prims=prims, steps=8,
                 lam=0.5, precision=prec, kahan=kahan)
        o = _oracle(2, 40, 24, O.PERIODIC, O.PERIODIC, prims=prims, steps=8,
                    lam=0.5)
        _assert_l1(g, o, 2)


@pytest.mark.parametrize("kahan", [1, 0])
def test_sod_1d_fp32_l1(kahan):
    g = _gpu(1, 1000, 1, L.TRANSMISSIVE, 0, riemann=SOD, steps=200,
             precision=L.F32, kahan=kahan)
    o = _oracle(1, 1000, 1, O.TRANSMISSIVE, 0, riemann=SOD, steps=200)
    _assert_l1(g, o, 1)


@pytest.mark.parametrize("kahan", [1, 0])
@pytest.mark.parametrize("bcs", BC2)
def test_random_2d_fp32_l1(bcs, kahan):
    """The deposit kernel, compensated (kahan = 1) and plain (kahan = 0):
    one-type tiles in the first kernel, mixed windows in the second (this
    smooth field with a jump has both)."""
    nx, ny = 70, 45
    prims = I.random_smooth_prims(2, nx, ny, seed=3000 + bcs[0])
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=20, precision=L.F32,
             kahan=kahan)
    o = _oracle(2, nx, ny, *bcs, prims=prims, steps=20)
    _assert_l1(g, o, 2)


@pytest.mark.parametrize("kahan", [1, 0])
def test_xonly_strong_jump_fp32_rows_identical(kahan):
    """x-only data whose level c1 changes across the jump (c1 = 1 | 0: mixed
    tiles on the general path) between reflecting walls: rows stay identical
    bit for bit and m_y stays zero, and the rows match the oracle's x-only
    run.  (Much stronger jumps make the square-lattice step chaotic even for
    x-only data - a 1e-12 perturbation reaches O(1) - so no two
    implementations can agree there.)"""
    nx, ny = 300, 70
    riem = ((1.0, 0.0, 1.0), (1.0, 0.0, 0.3), 0, 0.5, 0.5, 0.0)
    g = _gpu(2, nx, ny, L.TRANSMISSIVE, L.REFLECTING, riemann=riem, steps=150,
             precision=L.F32, kahan=kahan)
    for f in FIELDS:
        rows = g[f].reshape(ny, nx)
        assert np.array_equal(rows, np.broadcast_to(rows[0], rows.shape)), f
    assert np.all(g["my"] == 0.0)
    o = _oracle(2, nx, 1, O.TRANSMISSIVE, O.REFLECTING, riemann=riem,
                steps=150)
    row = {f: g[f].reshape(ny, nx)[0] for f in FIELDS}
    _assert_l1(row, o, 2)


@pytest.mark.parametrize("kahan", [1, 0])
def test_uniform_state_fp32_bitwise(kahan):
    n = 96
    prims = [np.full(n * n, 0.8), np.full(n * n, 0.37), np.full(n * n, -0.61),
             np.full(n * n, 0.9)]
    g = _gpu(2, n, n, L.PERIODIC, L.PERIODIC, prims=prims, steps=25,
             precision=L.F32, kahan=kahan)
    for f in FIELDS:
        assert np.all(g[f] == g[f][0])


def test_sod_2d_full_size_rows_match_oracle():
    """4096 x 512 square lattice, x-only Sod jump, transmissive x,
    reflecting y, to t = 0.2 (820 steps): every row is identical on the GPU
    and equals (bit for bit in FP64) the oracle's single-row run between the
    same reflecting walls, which by the mirror construction is the same
    x-only solution."""
    nx, ny = 4096, 512
    n, lam = O.steps_and_lambda(0.2, 1.0 / nx)
    o = _oracle(2, nx, 1, O.TRANSMISSIVE, O.REFLECTING, riemann=SOD, steps=n,
                lam=lam)
    for prec, kahan in ((L.F64, 1), (L.F32, 1), (L.F32, 0)):
        g = _gpu(2, nx, ny, L.TRANSMISSIVE, L.REFLECTING, riemann=SOD,
                 steps=n, lam=lam, precision=prec, kahan=kahan)
        for f in FIELDS:
            rows = g[f].reshape(ny, nx)
            assert np.array_equal(rows, np.broadcast_to(rows[0], rows.shape))
        row = {f: g[f].reshape(ny, nx)[0] for f in FIELDS}
        row["p"] = g["p"].reshape(ny, nx)[0]
        if prec == L.F64:
            _assert_bitwise(row, o, 2)
        else:
            _assert_l1(row, o, 2)


def _cylinder_patch_oracle(N, ix, iy, h, steps, cx=0.5, cy=0.5, r=0.4):
    """The oracle's value at node (ix, iy) of the N x N periodic cylinder
    after `steps` steps, from a (2h+1)^2 patch around it (periodic wrap of
    the indices).  The node's arrivals come from sources within the reach,
    in an order fixed relative to the node, so with h at least (steps + 1)
    reaches the patch's own (transmissive) edges cannot reach the centre
    and the value equals the full grid's."""
    dx = 1.0 / N
    x = O.node_x(N, 0.0, 1.0)
    y = 0.0 + (np.arange(N) + 0.5) * dx
    jx = np.take(np.arange(N), np.arange(ix - h, ix + h + 1), mode="wrap")
    jy = np.take(np.arange(N), np.arange(iy - h, iy + h + 1), mode="wrap")
    X, Y = np.meshgrid(x[jx], y[jy])
    r2 = (X - cx) * (X - cx) + (Y - cy) * (Y - cy)
    w = 2 * h + 1
    P = O.Params(dim=2, nx=w, ny=w, bc_x=O.TRANSMISSIVE, bc_y=O.TRANSMISSIVE)
    st = O._assign(P, (r2 < r * r).ravel(), (1.0, 0.0, 0.0, 1.0),
                   (0.125, 0.0, 0.0, 0.1), 1.0)
    st2, _ = O.run(P, st, steps)
    ph = O.lattice_to_physical(1.4, 1.0, st2)
    c = h * w + h
    return {f: ph[f][c] for f in FIELDS}


def test_cylinder_full_size_sampled_outputs():
    """The 8192^2 periodic cylinder at full size, two steps: sampled nodes
    (the centre, the circle's edge, the periodic corners, seeded others)
    against the oracle run on a patch around each.  FP64 bit for bit; the
    FP32 deposit kernel, plain and compensated, within 1e-5 of the field's
    range."""
    N, steps, h = 8192, 2, 24
    rng = np.random.default_rng(20263)
    edge = int(round((0.5 + 0.4) * N - 0.5))
    picks = [(N // 2, N // 2), (edge, N // 2), (N // 2, edge), (0, 0),
             (N - 1, N - 1), (0, N - 1)]
    picks += [tuple(int(v) for v in rng.integers(0, N, 2)) for _ in range(10)]
    ref = {(ix, iy): _cylinder_patch_oracle(N, ix, iy, h, steps)
           for ix, iy in picks}
    riem = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 1, 0.5, 0.5, 0.4)
    # field ranges after two steps (oracle, 512^2 and 96^2 alike)
    span = {"rho": 0.875, "mx": 0.777, "my": 0.777, "rhoE": 2.25}
    for prec, kahan in ((L.F64, 1), (L.F32, 0), (L.F32, 1)):
        g = _gpu(2, N, N, L.PERIODIC, L.PERIODIC, riemann=riem, steps=steps,
                 precision=prec, kahan=kahan)
        assert g["diag"]["flags"] == 0
        for (ix, iy), o in ref.items():
            k = iy * N + ix
            for f in FIELDS:
                if prec == L.F64:
                    assert g[f][k] == o[f], (prec, ix, iy, f, g[f][k], o[f])
                else:
                    assert abs(g[f][k] - o[f]) <= 1e-5 * span[f], (
                        prec, kahan, ix, iy, f, g[f][k], o[f])
        del g


def test_conservation_periodic_gpu():
    nx, ny = 96, 40
    prims = I.random_smooth_prims(2, nx, ny, seed=44, jump=False)
    for prec, tol, kahan in ((L.F64, 1e-13, 1), (L.F32, 1e-6, 1),
                             (L.F32, 1e-6, 0)):
        cfg = L.make_config(2, nx, ny, precision=prec, bc_x=L.PERIODIC,
                            bc_y=L.PERIODIC, kahan=kahan)
        with L.Solver(cfg) as s:
            s.set_primitives(*prims)
            t0 = s.conservation()
            s.step(200)
            t1 = s.conservation()
        scale = np.array([t0[0], t0[0], t0[0], t0[3]])
        assert np.all(np.abs(t1 - t0) <= tol * scale), (prec, (t1 - t0) / scale)


@pytest.mark.parametrize("n", [1000, 5000, 200000])
def test_conservation_periodic_1d_gpu(n):
    """Periodic 1-D tubes (16-, 32- and 256-node tiles): the device totals
    of mass and energy do not drift, and equal the sums of the state read
    back (FP32: compensated FP32 sums of the nodes; FP64: FP64 sums)."""
    prims = I.random_smooth_prims(1, n, 1, seed=45 + n, jump=False)
    for prec, tol, kahan in ((L.F64, 1e-13, 1), (L.F32, 1e-6, 1),
                             (L.F32, 1e-6, 0)):
        cfg = L.make_config(1, n, precision=prec, bc_x=L.PERIODIC, kahan=kahan)
        with L.Solver(cfg) as s:
            s.set_primitives(*prims)
            t0 = s.conservation()
            s.step(100)
            t1 = s.conservation()
            m = s.moments()
        scale = np.array([t0[0], t0[0], 1.0, t0[3]])
        assert np.all(np.abs(t1 - t0) <= tol * scale), (prec, (t1 - t0) / scale)
        rel = 1e-12 if prec == L.F64 else 1e-9
        assert abs(t1[0] - np.sum(m["rho"])) <= rel * t1[0], (prec, kahan)


def test_restart_bitwise():
    """Checkpoint through lbm_moments / lbm_set_moments: n then m steps
    equal n + m steps (FP64, lambda = 1 so the unit conversion is exact)."""
    prims = I.random_smooth_prims(2, 50, 30, seed=5)
    cfg = L.make_config(2, 50, 30, bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING)
    with L.Solver(cfg) as a:
        a.set_primitives(*prims)
        a.step(12)
        ref = a.moments()
    with L.Solver(cfg) as b:
        b.set_primitives(*prims)
        b.step(5)
        m = b.moments()
        b.set_moments(m["rho"], m["mx"], m["my"], m["rhoE"])
        b.step(7)
        got = b.moments()
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f])


def test_errors_are_reported():
    with pytest.raises(L.LbmError) as e:
        L.Solver(L.make_config(3, 10))
    assert e.value.status == L.EINVAL
    # negative density in the input: reported as LBM_ESTATE
    cfg = L.make_config(1, 64, bc_x=L.PERIODIC)
    with L.Solver(cfg) as s:
        rho = np.ones(64)
        rho[5] = -1.0
        with pytest.raises(L.LbmError) as e:
            s.set_primitives(rho, np.zeros(64), None, np.ones(64))
            s.step(1)
            s.moments()
        assert e.value.status == L.ESTATE
    # reach beyond max_reach: state untouched, LBM_EREACH
    cfg = L.make_config(1, 64, bc_x=L.PERIODIC, max_reach=2)
    with L.Solver(cfg) as s:
        s.set_primitives(np.ones(64), np.zeros(64), None, np.ones(64))
        s.step(1)
        with pytest.raises(L.LbmError) as e:
            s.synchronize()
        assert e.value.status == L.EREACH


@pytest.mark.parametrize("prec,kahan", [(L.F64, 1), (L.F32, 1), (L.F32, 0)])
def test_errors_are_reported_2d(prec, kahan):
    """Square lattice, every step path (FP64 records pass and gather, FP32
    deposit kernel plain and compensated): a negative density is
    LBM_ESTATE; a reach beyond max_reach is LBM_EREACH."""
    n = 40
    N = n * n
    cfg = L.make_config(2, n, n, precision=prec, kahan=kahan,
                        bc_x=L.PERIODIC, bc_y=L.PERIODIC)
    with L.Solver(cfg) as s:
        rho = np.ones(N)
        rho[123] = -1.0
        with pytest.raises(L.LbmError) as e:
            s.set_primitives(rho, np.zeros(N), np.zeros(N), np.ones(N))
            s.step(1)
            s.moments()
        assert e.value.status == L.ESTATE
    # c1 = 1 at rest gives reach 3: a limit of 2 is exceeded
    cfg = L.make_config(2, n, n, precision=prec, kahan=kahan,
                        bc_x=L.PERIODIC, bc_y=L.PERIODIC, max_reach=2)
    with L.Solver(cfg) as s:
        s.set_primitives(np.ones(N), np.zeros(N), np.zeros(N), np.ones(N))
        s.step(1)
        with pytest.raises(L.LbmError) as e:
            s.synchronize()
        assert e.value.status == L.EREACH


def test_uniform_state_stays_uniform_bitwise():
    n = 64
    for dim in (1, 2):
        N = n * (n if dim == 2 else 1)
        prims = [np.full(N, 0.8), np.full(N, 0.37),
                 np.full(N, -0.61) if dim == 2 else None, np.full(N, 0.9)]
        g = _gpu(dim, n, n if dim == 2 else 1, L.PERIODIC, L.PERIODIC,
                 prims=prims, steps=25)
        for f in FIELDS:
            if f == "my" and dim == 1:
                continue
            assert np.all(g[f] == g[f][0])


def test_restart_fp32_records_bitwise():
    """FP32 square lattice: checkpoint through lbm_moments / lbm_set_moments
    in the same handle (its per-tile window records carry on): n then m
    steps must equal n + m steps bit for bit (lambda = 1, so the unit
    conversion is exact)."""
    nx, ny = 77, 45
    prims = I.random_smooth_prims(2, nx, ny, seed=71)
    cfg = L.make_config(2, nx, ny, precision=L.F32, bc_x=L.TRANSMISSIVE,
                        bc_y=L.REFLECTING, kahan=0)
    with L.Solver(cfg) as a:
        a.set_primitives(*prims)
        a.step(13)
        ref = a.moments()
    with L.Solver(cfg) as b:
        b.set_primitives(*prims)
        for part in (4, 6, 3):
            b.step(part)
            m = b.moments()
            b.set_moments(m["rho"], m["mx"], m["my"], m["rhoE"])
        got = b.moments()
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f


@pytest.mark.parametrize("prec,kahan", [(L.F64, 1), (L.F32, 1), (L.F32, 0)])
def test_energy_clamps_counted_like_oracle(prec, kahan):
    """Nodes whose internal energy e = E - |V|^2/2 is negative are clamped to
    e = 0 and counted once per step that uses them, by every kernel (the
    FP32 deposit kernel counts them in the walk that owns the node)."""
    nx, ny = 48, 40
    n = nx * ny
    rng = np.random.default_rng(8)
    rho = rng.uniform(0.5, 1.5, n)
    u = rng.uniform(-0.4, 0.4, n)
    v = rng.uniform(-0.4, 0.4, n)
    rhoE = rho * (0.5 * (u * u + v * v) + rng.uniform(0.3, 0.8, n))
    bad = rng.choice(n, 37, replace=False)
    rhoE[bad] = 0.5 * rho[bad] * (u[bad] ** 2 + v[bad] ** 2) * 0.5
    cfg = L.make_config(2, nx, ny, precision=prec, bc_x=L.PERIODIC,
                        bc_y=L.PERIODIC, kahan=kahan)
    with L.Solver(cfg) as s:
        s.set_moments(rho, rho * u, rho * v, rhoE)
        s.step(1)
        d = s.diagnostics()
    P = O.Params(dim=2, nx=nx, ny=ny, bc_x=O.PERIODIC, bc_y=O.PERIODIC)
    st = O.State(rho.copy(), (rho * u).copy(), (rho * v).copy(), rhoE.copy())
    _, ec = O.run(P, st, 1)
    assert ec == 37
    assert d["eclamps"] == ec


def test_fp32_deposit_kernel_reports_bad_state():
    nx, ny = 64, 40
    cfg = L.make_config(2, nx, ny, precision=L.F32, bc_x=L.PERIODIC,
                        bc_y=L.PERIODIC, kahan=0)
    with L.Solver(cfg) as s:
        rho = np.ones(nx * ny)
        rho[700] = -1.0
        z = np.zeros(nx * ny)
        with pytest.raises(L.LbmError) as e:
            s.set_primitives(rho, z, z, np.ones(nx * ny))
            s.step(1)
            s.moments()
        assert e.value.status == L.ESTATE


@pytest.mark.parametrize("bcs", BC2)
@pytest.mark.parametrize("shape", [(3, 2), (7, 5), (33, 9)])
def test_tiny_grids_fp32_deposit_kernel(bcs, shape):
    """Grids narrower than the migration halo: most window slots of the
    deposit kernel lie outside the grid and are filled from the nodes that
    supply them (possibly several reflections or wraps away).  Mean error
    within 1e-5 of the field's range (the stated metric) wherever that
    range is at least 1 % of the field's size.  On a 3 x 2 grid a field may
    vary by only 1e-4 of its size, and m_y between two walls one row apart
    is a near-cancelling sum of O(1) terms; there the error is taken
    relative to the field's size (momentum: the larger of max |m_x| and max
    |m_y|): a slot filled from the wrong node or with the wrong mirror sign
    errs by the size of its contribution itself."""
    nx, ny = shape
    prims = I.random_smooth_prims(2, nx, ny, seed=4100 + nx * ny + bcs[0])
    g = _gpu(2, nx, ny, *bcs, prims=prims, steps=8, precision=L.F32,
             kahan=0)
    o = _oracle(2, nx, ny, *bcs, prims=prims, steps=8)
    mom = max(np.max(np.abs(o["mx"])), np.max(np.abs(o["my"])))
    for f in FIELDS:
        size = mom if f in ("mx", "my") else np.max(np.abs(o[f]))
        rng = np.ptp(o[f])
        scale = rng if rng >= 1e-2 * size else max(size, 1e-300)
        err = np.mean(np.abs(g[f] - o[f])) / scale
        assert err <= 1e-5, (f, err, rng, size)


def test_sod_1d_solve_replayed_from_cuda_graph_bitwise():
    """A whole solve (initial state + 200 steps, FP64) captured through the
    C ABI into one CUDA graph: every replay gives the oracle's result bit
    for bit (the step's device state - reach, flags, ticket - is reset by
    the solve itself, so replays do not drift)."""
    import torch
    stream = torch.cuda.Stream()
    cfg = L.make_config(1, 1000, precision=L.F64, bc_x=L.TRANSMISSIVE,
                        stream=stream.cuda_stream)
    o = _oracle(1, 1000, 1, O.TRANSMISSIVE, 0, riemann=SOD, steps=200)
    with L.Solver(cfg) as s:
        def solve():
            s.init_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), L.PLANAR_X,
                           0.5)
            s.step(200)
        with torch.cuda.stream(stream):
            solve()  # warm-up outside capture
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            solve()
        for _ in range(2):
            with torch.cuda.stream(stream):
                g.replay()
            stream.synchronize()
            m = s.moments()
            for f in ("rho", "mx", "rhoE"):
                assert np.array_equal(m[f], o[f]), f


def test_fma_peak_measurement():
    """lbm_measure_fma_peak reports this GPU's FP32 and FP64 FMA rates: both
    positive, FP32 far above FP64 on a GB300 (FP64 runs at a small fraction
    of the FP32 rate), and bad arguments are rejected."""
    p32 = L.lbm_measure_fma_peak(L.F32)
    p64 = L.lbm_measure_fma_peak(L.F64)
    assert 1e12 < p32 < 1e15 and 1e10 < p64 < 1e14
    assert p32 > 8 * p64
    with pytest.raises(L.LbmError) as e:
        L.lbm_measure_fma_peak(7)
    assert e.value.status == L.EINVAL


def test_fp32_reciprocal_and_quotient_against_correct_rounding():
    """The FP32 kernels' reciprocal (hardware estimate + one Newton-Raphson
    step) is within one unit in the last place of the correctly rounded 1/x,
    and their quotient by the level denominators 4 (2 c1 + 1) (eqs 24-25,
    Markstein's correction) within one of the correctly rounded n / d, over
    a million generated inputs each."""
    w_rcp, w_div = L.lbm_check_fp32_arith(1 << 20, seed=2026)
    assert w_rcp <= 1.0, w_rcp
    assert w_div <= 1.0, w_div
    with pytest.raises(L.LbmError):
        L.lbm_check_fp32_arith(-1)


@pytest.mark.parametrize("prec,kahan", [(L.F32, 0), (L.F32, 1), (L.F64, 1)])
def test_step_totals_match_exact_sum_of_the_state(prec, kahan):
    """The totals the step kernels form while stepping (a10: compensated
    FP32 pairs converted to FP64 once in the FP32 kernels, FP64 in the FP64
    kernels) against the exactly rounded sum (math.fsum) of the same state
    read back: within 1e-12 of the sum of magnitudes, on a grid of several
    tiles with ragged edges."""
    import math
    nx, ny = 300, 170
    prims = I.random_smooth_prims(2, nx, ny, seed=4100)
    cfg = L.make_config(2, nx, ny, precision=prec, bc_x=L.PERIODIC,
                        bc_y=L.PERIODIC, kahan=kahan, cons_every=1)
    with L.Solver(cfg) as s:
        s.set_primitives(*prims)
        s.step(7)
        tot = s.last_totals()
        g = s.moments()
    for k, f in enumerate(FIELDS):
        want = math.fsum(g[f].tolist())
        scale = math.fsum(np.abs(g[f]).tolist())
        assert abs(tot[k] - want) <= 1e-12 * scale, (f, tot[k], want, scale)
