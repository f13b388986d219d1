"""Invariants of the tau = 1 step that hold at any size, used to pin the
oracle: conservation, uniform states, the pressure flux of a shock tube,
the 2-D / 1-D relations of Section V.D, lattice symmetries, restart."""
import numpy as np
import pytest

from oracle import oracle as O, riemann as Rm

SOD_L = (1.0, 0.0, 1.0)
SOD_R = (0.125, 0.0, 0.1)
G = 1.4


def _random_smooth(P, seed, vmax=0.9):
    rng = np.random.default_rng(seed)
    nx, ny = P.nx, (P.ny if P.dim == 2 else 1)
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)
    ph = rng.uniform(0, 2 * np.pi, 6)
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
    u = vmax * np.sin(2 * np.pi * X + ph[2])
    v = vmax * np.cos(2 * np.pi * Y + ph[3]) if P.dim == 2 else None
    p = 1.0 + 0.6 * np.cos(2 * np.pi * (X + Y) + ph[4])
    return O.prims_to_lattice(G, 1.0, rho.ravel(), u.ravel(),
                              None if v is None else v.ravel(), p.ravel())


@pytest.mark.parametrize("dim,shape,steps", [(1, (64,), 1000),
                                             (2, (20, 16), 200)])
def test_periodic_conservation(dim, shape, steps):
    """Eq 22 per node plus periodic migration: total mass, momentum and
    energy are constant to round-off."""
    P = O.Params(dim=dim, nx=shape[0], ny=shape[1] if dim == 2 else 1,
                 bc_x=O.PERIODIC, bc_y=O.PERIODIC)
    s = _random_smooth(P, 3 + dim)
    t0 = O.totals(s)
    s2, _ = O.run(P, s, steps)
    t1 = O.totals(s2)
    scale = np.array([t0[0], np.abs(s.rho).sum(), np.abs(s.rho).sum(), t0[3]])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def test_reflecting_box_conserves_mass_energy():
    """Mirrored packets keep their mass and energy; only the normal momentum
    flips, so a closed box conserves mass and energy."""
    P = O.Params(dim=2, nx=18, ny=14, bc_x=O.REFLECTING, bc_y=O.REFLECTING)
    s = _random_smooth(P, 9)
    t0 = O.totals(s)
    s2, _ = O.run(P, s, 150)
    t1 = O.totals(s2)
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
    assert abs(t1[3] - t0[3]) <= 1e-13 * t0[3]


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("state", [(1.0, 0.37, -0.61, 1.0),   # fractional V
                                   (0.8, 1.25, 0.5, 0.05),    # c1 = 0
                                   (2.0, -1.7, 2.3, 9.0)])    # c1 >= 2
def test_uniform_state_stays_uniform(dim, state):
    rho, u, v, p = state
    n = 24
    P = O.Params(dim=dim, nx=n, ny=n if dim == 2 else 1, bc_x=O.PERIODIC,
                 bc_y=O.PERIODIC)
    N = n * (n if dim == 2 else 1)
    s = O.prims_to_lattice(G, 1.0, np.full(N, rho), np.full(N, u),
                           np.full(N, v) if dim == 2 else None, np.full(N, p))
    steps = 5
    s2, _ = O.run(P, s, steps)
    # round-off only: at most ~1e-14 relative per step (32 landings summed)
    for a, b in zip(s.fields(), s2.fields()):
        assert np.max(np.abs(a - b)) <= steps * 1e-14 * max(np.max(np.abs(a)),
                                                            rho)


def test_sod_momentum_grows_by_pressure_jump():
    """Transmissive ends with both end states at rest: mass and energy are
    constant and the total lattice momentum grows by exactly
    (p_L - p_R) lambda^2 per step (the momentum flux of eq 17 through each
    end), until a wave reaches an end."""
    N = 400
    P = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    lam = 1.0
    s = O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam)
    t0 = O.totals(s)
    for k in range(1, 41):
        s, _, _ = O.step(P, s)
        t = O.totals(s)
        assert abs(t[0] - t0[0]) <= 1e-13 * t0[0]
        assert abs(t[3] - t0[3]) <= 1e-13 * t0[3]
        assert t[1] == pytest.approx(k * (1.0 - 0.1) * lam * lam, rel=1e-12)


def _run_2d_xonly(nx, ny, bc_y, t_end=0.2):
    P = O.Params(dim=2, nx=nx, ny=ny, bc_x=O.TRANSMISSIVE, bc_y=bc_y)
    n, lam = O.steps_and_lambda(t_end, 1.0 / nx)
    s = O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam)
    s2, _ = O.run(P, s, n)
    return P, s2, lam


@pytest.mark.parametrize("bc_y", [O.PERIODIC, O.REFLECTING])
def test_xonly_2d_rows_identical(bc_y):
    """Section V.C's 400x4 lattice: data varying only along x stays so, bit
    for bit, and carries no y-momentum.  Any seed of row-to-row difference
    would grow: the square-lattice step amplifies transverse perturbations."""
    P, s, lam = _run_2d_xonly(400, 4, bc_y)
    for f in (s.rho, s.mx, s.rhoE):
        F = f.reshape(4, 400)
        assert np.array_equal(F, np.broadcast_to(F[0], F.shape))
    assert np.all(s.my == 0.0)


def test_square_lattice_amplifies_transverse_noise():
    """A property of the square-lattice step itself, recorded so that the
    summation-order reading above stays justified: a uniform gas at rest,
    perturbed at 1e-9, grows by orders of magnitude within 40 steps, while
    the 1-D lattice damps the same perturbation."""
    def grow(dim):
        n = 16
        P = O.Params(dim=dim, nx=n, ny=n if dim == 2 else 1, bc_x=O.PERIODIC,
                     bc_y=O.PERIODIC)
        N = n * (n if dim == 2 else 1)
        s = O.prims_to_lattice(G, 1.0, np.ones(N), np.zeros(N),
                               np.zeros(N) if dim == 2 else None, np.ones(N))
        rng = np.random.default_rng(1)
        s.rho = s.rho * (1 + 1e-9 * rng.standard_normal(N))
        a0 = np.abs(s.rho - s.rho.mean()).max()
        s, _ = O.run(P, s, 40)
        return np.abs(s.rho - s.rho.mean()).max() / a0
    assert grow(2) > 100.0
    assert grow(1) < 1.0


def projected_1d_step(rho, m, E, gamma, ghost=8):
    """Independent numpy restatement of one square-lattice step for data
    that varies only along x, projected onto x: per level v, two packets
    move by +-c_v along x and the two y-packets stay at x-offset 0, all with
    mass d_v; D = 2 in eqs 15 and 24-26; zero-gradient ghosts at both ends."""
    n = len(rho)
    pad = lambda a: np.concatenate([np.full(ghost, a[0]), a,
                                    np.full(ghost, a[-1])])
    r, mm, ee = pad(rho), pad(m), pad(E)
    V = mm / r
    e = ee / r - 0.5 * V * V
    e = np.maximum(e, 0.0)
    Q = 2.0 * (gamma - 1.0) * r * e
    c1 = np.floor(np.sqrt(Q / r)).astype(np.int64)
    c2 = c1 + 1
    d1 = (c2 ** 2 * r - Q) / (4.0 * (c2 ** 2 - c1 ** 2))
    d2 = (Q - c1 ** 2 * r) / (4.0 * (c2 ** 2 - c1 ** 2))
    phi = (1.0 - (gamma - 1.0)) * e
    nV = np.floor(V).astype(np.int64)
    f = V - nV
    out = np.zeros((3, n))
    xs = np.arange(len(r)) - ghost
    for d, c in ((d1, c1), (d2, c2)):
        for off, cb, zeta in ((c, V + c, None), (-c, V - c, None),
                              (0 * c, V, "y"), (0 * c, V, "y")):
            if zeta is None:
                en = 0.5 * cb * cb + phi
            else:
                en = 0.5 * (V * V + c * c) + phi
            for k, w in ((0, 1.0 - f), (1, f)):
                L = xs + nV + off + k
                ok = (L >= 0) & (L < n)
                np.add.at(out[0], L[ok], (w * d)[ok])
                np.add.at(out[1], L[ok], (w * d * cb)[ok])
                np.add.at(out[2], L[ok], (w * d * en)[ok])
    return out


def test_2d_rows_equal_projected_1d_scheme():
    """Every row of the x-only 2-D run equals an independent 1-D run of the
    x-projected square-lattice velocity set."""
    nx, ny = 200, 4
    P = O.Params(dim=2, nx=nx, ny=ny, bc_x=O.TRANSMISSIVE, bc_y=O.PERIODIC)
    n, lam = O.steps_and_lambda(0.2, 1.0 / nx)
    s = O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam)
    r, m, E = s.rho[:nx].copy(), s.mx[:nx].copy(), s.rhoE[:nx].copy()
    for _ in range(n):
        s, _, _ = O.step(P, s)
        r, m, E = projected_1d_step(r, m, E, G)
        for f2, f1 in ((s.rho, r), (s.mx, m), (s.rhoE, E)):
            rows = f2.reshape(ny, nx)
            assert np.max(np.abs(rows - f1)) <= 1e-12 * np.max(np.abs(f1))


def test_1d_and_2d_agree_to_discretisation_level():
    """Section V.D: the 1-D and 2-D schemes give the same profiles, both close
    to the analytical solution; their difference is no larger than the larger
    of their errors against it."""
    N = 400
    P1 = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    n, lam = O.steps_and_lambda(0.2, 1.0 / N)
    s1, _ = O.run(P1, O.riemann_planar(P1, 0, 1, 0.5, SOD_L, SOD_R, lam), n)
    P2, s2, _ = _run_2d_xonly(N, 4, O.PERIODIC)
    x = O.node_x(N, 0, 1)
    ph1 = O.lattice_to_physical(G, lam, s1)
    ph2 = O.lattice_to_physical(G, lam, O.State(s2.rho[:N], s2.mx[:N], None,
                                                s2.rhoE[:N]))
    for k in ("rho", "u", "p"):
        e1 = Rm.l1_errors(x, 0.2, 0.5, SOD_L, SOD_R, ph1["rho"], ph1["u"],
                          ph1["p"])[k]
        e2 = Rm.l1_errors(x, 0.2, 0.5, SOD_L, SOD_R, ph2["rho"], ph2["u"],
                          ph2["p"])[k]
        diff = float(np.mean(np.abs(ph1[k] - ph2[k])))
        assert diff <= max(e1, e2), (k, diff, e1, e2)


@pytest.mark.parametrize("bc", [O.PERIODIC, O.TRANSMISSIVE, O.REFLECTING])
def test_transpose_symmetry(bc):
    """The square lattice treats x and y alike: a jump along y evolves into
    the transpose of the same jump along x."""
    n = 20
    P = O.Params(dim=2, nx=n, ny=n, bc_x=bc, bc_y=bc)
    s = O.riemann_planar(P, 0, 1, 0.37, (1.0, 0.3, -0.2, 1.0),
                         (0.2, -0.1, 0.4, 0.15), 1.0)
    r = s.rho.reshape(n, n)
    sT = O.State(r.T.ravel().copy(), s.my.reshape(n, n).T.ravel().copy(),
                 s.mx.reshape(n, n).T.ravel().copy(),
                 s.rhoE.reshape(n, n).T.ravel().copy())
    a, _ = O.run(P, s, 8)
    b, _ = O.run(P, sT, 8)
    T = lambda f: f.reshape(n, n).T.ravel()
    for fa, fb in ((a.rho, b.rho), (a.mx, b.my), (a.my, b.mx),
                   (a.rhoE, b.rhoE)):
        assert np.max(np.abs(T(fa) - fb)) <= 1e-14 * np.max(np.abs(fa))


def test_cylinder_keeps_square_symmetry():
    """A centred circular Riemann problem on a periodic square keeps the
    symmetries of the square (reflections in x, y and the diagonal)."""
    n = 32
    P = O.Params(dim=2, nx=n, ny=n, bc_x=O.PERIODIC, bc_y=O.PERIODIC)
    s = O.riemann_circle(P, 0, 1, 0, 0.5, 0.5, 0.25, (1.0, 0.0, 0.0, 1.0),
                         (0.125, 0.0, 0.0, 0.1), 1.0)
    s2, _ = O.run(P, s, 12)
    r = s2.rho.reshape(n, n)
    mx = s2.mx.reshape(n, n)
    my = s2.my.reshape(n, n)
    E = s2.rhoE.reshape(n, n)
    tol = 1e-13
    sc = np.max(np.abs(r))
    assert np.max(np.abs(r - r[:, ::-1])) <= tol * sc
    assert np.max(np.abs(r - r[::-1, :])) <= tol * sc
    assert np.max(np.abs(r - r.T)) <= tol * sc
    assert np.max(np.abs(E - E.T)) <= tol * np.max(E)
    assert np.max(np.abs(mx + mx[:, ::-1])) <= tol * sc
    assert np.max(np.abs(mx - my.T)) <= tol * sc


def test_restart_composes():
    """The state is the moments alone (eq 10 at tau = 1): n steps then m
    steps equal n + m steps bit for bit."""
    P = O.Params(dim=2, nx=16, ny=12, bc_x=O.TRANSMISSIVE, bc_y=O.REFLECTING)
    s = _random_smooth(P, 77)
    a, _ = O.run(P, s, 7)
    a, _ = O.run(P, a, 5)
    b, _ = O.run(P, s, 12)
    for fa, fb in zip(a.fields(), b.fields()):
        assert np.array_equal(fa, fb)


def test_stored_sod2d_row_is_the_oracle_solution():
    """The stored oracle row of the 4096 x 512 tube (written by
    tests/golden/make_golden.py) has one row per node and conserves mass:
    at t = 0.2 no wave has reached the transmissive ends, so the total is
    that of the initial state, 0.5 * 1 + 0.5 * 0.125."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden",
                        "sod2d_row_4096_t0.2.txt")
    a = np.loadtxt(path)
    assert a.shape == (4096, 3)
    np.testing.assert_allclose(a[:, 0].sum() / 4096, 0.5625, rtol=1e-13)
    assert a[0, 0] == 1.0 and a[-1, 0] == 0.125   # undisturbed ends
