"""Closed-form pins of the oracle's equilibrium (Section III.B, Section IV).

Each test checks a property the paper's equations fix exactly, so that a
dropped term, a wrong sign or a swapped operand in the oracle fails one of
them.
"""
import os
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sod_equilibria.txt")
GAMMA = 1.4


def _rows():
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("|")
        a = [F(t) for t in lhs.split()]
        b = [F(t) for t in rhs.split()]
        yield int(a[0]), a[1:], b


def _mass_by_speed(dim, c1, c2, d0, d1, d2):
    """Mass carried at each |c'| (what the packets physically are)."""
    out = {}
    b = 2 if dim == 1 else 4
    for c, m in ((0, d0), (c1, b * d1), (c2, b * d2)):
        out[c] = out.get(c, 0.0) + float(m)
    return {c: m for c, m in out.items() if abs(m) > 1e-15}


@pytest.mark.parametrize("row", list(_rows()), ids=lambda r: str(r[0]))
def test_hand_derived_equilibria(row):
    dim, (rho, mx, my, rhoE), (c1, c2, d0, d1, d2, phi) = row
    P = O.Params(dim=dim, nx=4, ny=4 if dim == 2 else 1, gamma=GAMMA)
    q = O.equilibrium(P, float(rho), float(mx), float(my), float(rhoE))
    assert q["phi"] == pytest.approx(float(phi), rel=1e-14)
    assert q["d0"] == pytest.approx(float(d0), rel=1e-14, abs=1e-16)
    got = _mass_by_speed(dim, q["c1"], q["c2"], q["d0"], q["d1"], q["d2"])
    want = _mass_by_speed(dim, int(c1), int(c2), d0, d1, d2)
    assert set(got) == set(want)
    for c in want:
        assert got[c] == pytest.approx(want[c], rel=1e-13)


def test_sod_levels_exact():
    """The Sod rows are far from any square: c1 must match exactly."""
    for dim, st, ref in list(_rows())[:4]:
        P = O.Params(dim=dim, nx=4, ny=4 if dim == 2 else 1, gamma=GAMMA)
        q = O.equilibrium(P, *(float(v) for v in st))
        assert (q["c1"], q["c2"]) == (int(ref[0]), int(ref[1]))
        assert q["d1"] == pytest.approx(float(ref[3]), rel=1e-14)
        assert q["d2"] == pytest.approx(float(ref[4]), rel=1e-13)


def _random_states(dim, n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.05, 5.0, n)
    V = rng.uniform(-3.0, 3.0, (n, 2))
    if dim == 1:
        V[:, 1] = 0.0
    e = np.exp(rng.uniform(np.log(0.01), np.log(40.0), n))
    m = rho[:, None] * V
    rhoE = rho * (e + 0.5 * (V ** 2).sum(1))
    return rho, m, rhoE, e, V


@pytest.mark.parametrize("dim", [1, 2])
def test_packets_reproduce_moments(dim):
    """Eq 22: the packets of a node sum to its own (rho, rho V, rho E)."""
    P = O.Params(dim=dim, nx=4, ny=4 if dim == 2 else 1, gamma=GAMMA)
    rho, m, rhoE, e, V = _random_states(dim, 300, 11 + dim)
    for i in range(len(rho)):
        pk = O.packets(P, rho[i], m[i, 0], m[i, 1], rhoE[i])
        assert pk.shape[0] == (5 if dim == 1 else 8)
        tot = pk[:, 2:].sum(0)
        assert tot[0] == pytest.approx(rho[i], rel=1e-13)
        assert tot[1] == pytest.approx(m[i, 0], rel=1e-12, abs=1e-13 * rho[i])
        assert tot[2] == pytest.approx(m[i, 1], rel=1e-12, abs=1e-13 * rho[i])
        assert tot[3] == pytest.approx(rhoE[i], rel=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_second_moment_is_pressure(dim):
    """Eq 17 with eq 27: sum m (c-V)(c-V) = (gamma-1) rho e I, i.e. the
    equilibrium carries the Euler momentum flux rho V V + P I."""
    P = O.Params(dim=dim, nx=4, ny=4 if dim == 2 else 1, gamma=GAMMA)
    rho, m, rhoE, e, V = _random_states(dim, 200, 21 + dim)
    for i in range(len(rho)):
        pk = O.packets(P, rho[i], m[i, 0], m[i, 1], rhoE[i])
        mass = pk[:, 2]
        cb = pk[:, 3:5] / mass[:, None]
        dev = cb - V[i]
        T = np.einsum("p,pa,pb->ab", mass, dev, dev)
        p = (GAMMA - 1.0) * rho[i] * e[i]
        assert T[0, 0] == pytest.approx(p, rel=1e-11)
        if dim == 2:
            assert T[1, 1] == pytest.approx(p, rel=1e-11)
            assert abs(T[0, 1]) <= 1e-11 * p


@pytest.mark.parametrize("dim", [1, 2])
def test_velocity_set_symmetry(dim):
    """Eqs 16-18 on each level: sum c' = 0, sum c'c' = (b_v/D) c_v^2 I,
    sum c'c'c' = 0."""
    P = O.Params(dim=dim, nx=4, ny=4 if dim == 2 else 1, gamma=GAMMA)
    rho, m, rhoE, e, V = _random_states(dim, 50, 31 + dim)
    b = 2 if dim == 1 else 4
    for i in range(len(rho)):
        pk = O.packets(P, rho[i], m[i, 0], m[i, 1], rhoE[i])
        c = pk[:, 0:2]
        speed = np.abs(c).max(1)
        levels = (pk[1:3], pk[3:5]) if dim == 1 else (pk[0:4], pk[4:8])
        for lv in levels:
            cv = lv[:, 0:2]
            assert len(cv) == b
            assert np.all(cv.sum(0) == 0)
            S2 = np.einsum("pa,pb->ab", cv, cv)
            cmag = np.abs(cv).max()
            assert np.allclose(S2[:dim, :dim], b / dim * cmag ** 2 * np.eye(dim))
            S3 = np.einsum("pa,pb,pc->abc", cv, cv, cv)
            assert np.all(S3 == 0)
        assert speed.max() <= np.abs(c).max()


@pytest.mark.parametrize("dim", [1, 2])
def test_levels_bracket_and_nonnegative(dim):
    """Eq 26 picks c1 so that c1^2 <= X < c2^2, which keeps d1, d2 >= 0."""
    P = O.Params(dim=dim, nx=4, ny=4 if dim == 2 else 1, gamma=GAMMA)
    rho, m, rhoE, e, V = _random_states(dim, 400, 41 + dim)
    for i in range(len(rho)):
        q = O.equilibrium(P, rho[i], m[i, 0], m[i, 1], rhoE[i])
        d0 = 0.5 * rho[i] if dim == 1 else 0.0
        X = dim * (GAMMA - 1) * rho[i] * q["e"] / (rho[i] - d0)
        assert q["c1"] ** 2 <= X * (1 + 1e-15) and X < q["c2"] ** 2
        assert q["c2"] == q["c1"] + 1
        assert q["d1"] >= -1e-15 * rho[i] and q["d2"] >= -1e-15 * rho[i]


@pytest.mark.parametrize("dim", [1, 2])
def test_split_moves_mass_centre_by_V(dim):
    """Eqs 28-29: linear / bilinear splitting keeps the centre of mass of
    every packet at its continuous end point, so one node's mass lands with
    its centre at x + V, and the spread about it is the velocity spread plus
    the split's f(1-f).  A swapped weight moves the centre to x + n + 1 - f."""
    n = 40
    P = O.Params(dim=dim, nx=n, ny=n if dim == 2 else 1, gamma=GAMMA,
                 bc_x=O.PERIODIC, bc_y=O.PERIODIC)
    N = n * (n if dim == 2 else 1)
    rng = np.random.default_rng(5 + dim)
    for _ in range(10):
        V = rng.uniform(-2.5, 2.5, 2) if dim == 2 else np.array(
            [rng.uniform(-2.5, 2.5), 0.0])
        rho0, e = rng.uniform(0.5, 2.0), rng.uniform(0.2, 6.0)
        s = O.State(np.zeros(N), np.zeros(N), np.zeros(N) if dim == 2 else None,
                    np.zeros(N))
        src = (n // 2) * (n if dim == 2 else 0) + n // 2
        s.rho[src] = rho0
        s.mx[src] = rho0 * V[0]
        if dim == 2:
            s.my[src] = rho0 * V[1]
        s.rhoE[src] = rho0 * (e + 0.5 * (V ** 2).sum())
        out, _, _ = O.step(P, s)
        idx = np.arange(N)
        x = idx % n
        y = idx // n if dim == 2 else np.zeros(N)
        M = out.rho.sum()
        assert M == pytest.approx(rho0, rel=1e-13)
        cx = (out.rho * x).sum() / M
        assert cx == pytest.approx(n // 2 + V[0], abs=1e-12)
        q = O.equilibrium(P, rho0, rho0 * V[0], rho0 * V[1], s.rhoE[src])
        spread = (GAMMA - 1) * e  # sum m c'^2 / rho per axis (eq 17)
        f = q["fx"]
        var_x = (out.rho * (x - cx) ** 2).sum() / M
        assert var_x == pytest.approx(spread + f * (1 - f), rel=1e-11)
        if dim == 2:
            cy = (out.rho * y).sum() / M
            assert cy == pytest.approx(n // 2 + V[1], abs=1e-12)
