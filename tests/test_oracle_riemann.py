"""The paper's own comparison (Section V.C-D): the shock tube against the
analytical Riemann solution.  First the exact solver is pinned to published
values, then the oracle's lattice Boltzmann solution is held to it."""
import os

import numpy as np
import pytest

from oracle import oracle as O, riemann as Rm
from tests.golden.make_golden import sod_l1

HERE = os.path.join(os.path.dirname(__file__), "golden")
SOD_L = (1.0, 0.0, 1.0)
SOD_R = (0.125, 0.0, 0.1)


def _kv(name):
    out = {}
    for line in open(os.path.join(HERE, name)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_exact_solver_matches_published_star_state():
    ref = _kv("sod_exact_star.txt")
    st = Rm.star_state(SOD_L, SOD_R)
    w = Rm.wave_speeds(SOD_L, SOD_R)
    assert st.p == pytest.approx(ref["p_star"], abs=6e-6)
    assert st.u == pytest.approx(ref["u_star"], abs=6e-6)
    assert st.rho_l == pytest.approx(ref["rho_star_left"], abs=6e-6)
    assert st.rho_r == pytest.approx(ref["rho_star_right"], abs=6e-6)
    assert w["right_head"] == pytest.approx(ref["shock_speed"], abs=6e-6)
    for key, sp in (("x_head_t0.2", w["left_head"]),
                    ("x_tail_t0.2", w["left_tail"]),
                    ("x_contact_t0.2", w["contact"]),
                    ("x_shock_t0.2", w["right_head"])):
        assert 0.5 + 0.2 * sp == pytest.approx(ref[key], abs=6e-5)


def test_exact_solution_satisfies_jump_conditions():
    """Rankine-Hugoniot across the right shock; pressure and velocity
    continuous across the contact; Riemann invariant across the fan."""
    st = Rm.star_state(SOD_L, SOD_R)
    g = 1.4
    S = Rm.wave_speeds(SOD_L, SOD_R)["right_head"]
    rr, ur, pr = SOD_R
    r2, u2, p2 = st.rho_r, st.u, st.p
    assert rr * (ur - S) == pytest.approx(r2 * (u2 - S), rel=1e-12)
    assert rr * (ur - S) ** 2 + pr == pytest.approx(r2 * (u2 - S) ** 2 + p2,
                                                    rel=1e-12)
    x = np.linspace(0.27, 0.48, 50)
    rho, u, p = Rm.sample(x, 0.2, 0.5, SOD_L, SOD_R)
    a = np.sqrt(g * p / rho)
    J = u + 2 * a / (g - 1)
    assert np.allclose(J, J[0], rtol=1e-12)
    assert np.allclose(p / rho ** g, p[0] / rho[0] ** g, rtol=1e-12)


def test_lb_converges_to_exact_solution():
    """The scheme is first order (Section I): the L1 error must fall as the
    lattice is refined, and stays at the values the oracle gave when frozen
    (10% margin)."""
    rows = [l.split() for l in open(os.path.join(HERE, "sod_l1_errors.txt"))
            if l.strip() and not l.startswith("#")]
    prev = None
    for N, *frozen in rows[:2]:  # N = 400, 1000 (4000 in the slow test)
        e = sod_l1(int(N))
        for k, f in zip(("rho", "u", "p"), frozen):
            assert e[k] <= 1.1 * float(f)
            assert e[k] >= 0.9 * float(f)
        if prev is not None:
            for k in ("rho", "u", "p"):
                assert e[k] < prev[k]
        prev = e
    # the paper's 400-node lattice already tracks the exact solution closely
    assert float(rows[0][1]) < 0.01


@pytest.mark.slow
def test_lb_converges_at_4000_nodes():
    rows = [l.split() for l in open(os.path.join(HERE, "sod_l1_errors.txt"))
            if l.strip() and not l.startswith("#")]
    e = sod_l1(4000)
    for k, f in zip(("rho", "u", "p"), rows[2][1:]):
        assert 0.9 * float(f) <= e[k] <= 1.1 * float(f)
        assert e[k] < float(rows[1][1 + ("rho", "u", "p").index(k)])


def test_wave_positions_at_t02():
    """The shock sits where the exact solution puts it: the density jump
    to the undisturbed right state is within a few cells of x = 0.8504."""
    N = 1000
    P = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    n, lam = O.steps_and_lambda(0.2, 1.0 / N)
    s, _ = O.run(P, O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam), n)
    x = O.node_x(N, 0, 1)
    rho = s.rho
    mid = 0.5 * (0.26557 + 0.125)
    i = np.where((rho[:-1] > mid) & (rho[1:] <= mid))[0]
    assert len(i) >= 1
    assert abs(x[i[-1]] - 0.8504) < 5.0 / N
