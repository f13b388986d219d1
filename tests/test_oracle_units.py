"""Pins of the oracle's unit conversion at lambda = dt/dx != 1.

The oracle steps in lattice units: V = u lambda, and energies per unit mass
(so the lattice pressure) scale with lambda^2.  Every other pin runs at
lambda = 1, where a wrong power of lambda in the conversion cannot show.
These tests hold the conversion to physics that does not depend on lambda:

* the Euler conservation laws: while no wave reaches an end of a tube with
  transmissive ends, the physical totals of mass, momentum and energy change
  at exactly the rate the fluxes of the two uniform end states give (for a
  uniform state the scheme's discrete fluxes are exact, eqs 16-18, 22);
* the exact Riemann solution (the paper's comparison, Section V.C-D): a run
  at lambda = 0.5 tracks it as closely as a run at lambda = 1 does;
* in lattice units, the momentum of a tube at rest grows per step by the
  lattice pressure jump (p_L - p_R) lambda^2.

The last test plants each wrong power of lambda in the oracle (on the CPU)
and checks that these pins catch it.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests.golden.make_golden import (LAMBDA_CASES, SOD_L, SOD_R,
                                      riemann_l1_at_lambda)

G = 1.4
HERE = os.path.join(os.path.dirname(__file__), "golden")


def _fluxes(left, right, gamma=G):
    """Physical fluxes (mass, momentum, energy) of the Euler equations for
    the left state minus those of the right state."""
    out = []
    for rho, u, p in (left, right):
        E = p / (gamma - 1.0) + 0.5 * rho * u * u
        out.append(np.array([rho * u, rho * u * u + p, u * (E + p)]))
    return out[0] - out[1]


def _physical_totals(s, lam, dx):
    ph = O.lattice_to_physical(G, lam, s)
    return np.array([ph["rho"].sum(), ph["mx"].sum(), ph["rhoE"].sum()]) * dx


def totals_follow_fluxes(case, lam, N=400, t_end=0.2):
    """Largest relative departure of the physical totals at t_end from
    totals(0) + t_end * (flux_L - flux_R)."""
    left, right, x_d = LAMBDA_CASES[case]
    P = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    dx = 1.0 / N
    n = int(round(t_end / (lam * dx)))
    s0 = O.riemann_planar(P, 0, 1, x_d, left, right, lam)
    s, _ = O.run(P, s0, n)
    want = _physical_totals(s0, lam, dx) + t_end * _fluxes(left, right)
    got = _physical_totals(s, lam, dx)
    return float(np.max(np.abs(got - want) / np.abs(want)))


def lattice_momentum_growth(lam, N=400, steps=30):
    """Largest relative departure of the lattice momentum after k steps
    from k (p_L - p_R) lambda^2, and of mass and energy from their start."""
    P = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    s = O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam)
    t0 = O.totals(s)
    worst = 0.0
    for k in range(1, steps + 1):
        s, _, _ = O.step(P, s)
        t = O.totals(s)
        want = k * (SOD_L[2] - SOD_R[2]) * lam * lam
        worst = max(worst, abs(t[1] - want) / want,
                    abs(t[0] - t0[0]) / t0[0], abs(t[3] - t0[3]) / t0[3])
    return worst


def _frozen_l1():
    out = {}
    for line in open(os.path.join(HERE, "riemann_l1_lambda_half.txt")):
        if line.strip() and not line.startswith("#"):
            case, N, *v = line.split()
            out[(case, int(N))] = dict(zip(("rho", "u", "p"), map(float, v)))
    return out


def l1_at_half_matches(case, N=400):
    """The run at lambda = 0.5 is as close to the exact solution as the
    frozen values say (10 % margin) and no worse than 1.5x the run at
    lambda = 1 of the same lattice."""
    e = riemann_l1_at_lambda(case, N, 0.5)
    frozen = _frozen_l1()[(case, N)]
    e1 = riemann_l1_at_lambda(case, N, 1.0)
    return all(0.9 * frozen[k] <= e[k] <= 1.1 * frozen[k] and
               e[k] <= 1.5 * e1[k] for k in ("rho", "u", "p"))


@pytest.mark.parametrize("lam", [1.0, 0.5, 0.25])
@pytest.mark.parametrize("case", ["sod", "toro1"])
def test_physical_totals_follow_end_state_fluxes(case, lam):
    assert totals_follow_fluxes(case, lam) <= 1e-13


@pytest.mark.parametrize("lam", [1.0, 0.5])
def test_lattice_momentum_grows_by_lattice_pressure_jump(lam):
    assert lattice_momentum_growth(lam) <= 1e-12


@pytest.mark.parametrize("case", ["sod", "toro1"])
def test_lambda_half_tracks_exact_solution(case):
    assert l1_at_half_matches(case)
    # and converges under refinement at that lambda
    f = _frozen_l1()
    for k in ("rho", "u", "p"):
        assert f[(case, 1000)][k] < f[(case, 400)][k]


# --- planted mistakes: each wrong power of lambda must be caught -----------

def _prims_to_lattice_wrong(kind):
    def conv(gamma, lam, rho, u, v, p):
        rho = np.asarray(rho, dtype=np.float64)
        lv = lam * lam if kind == "velocity" else lam
        lp = lam if kind == "pressure" else lam * lam
        Vx = np.asarray(u, dtype=np.float64) * lv
        Vy = None if v is None else np.asarray(v, dtype=np.float64) * lv
        kin = Vx * Vx if Vy is None else Vx * Vx + Vy * Vy
        rhoE = np.asarray(p, dtype=np.float64) * lp / (gamma - 1.0) + 0.5 * rho * kin
        return O.State(rho.copy(), rho * Vx, None if Vy is None else rho * Vy,
                       rhoE)
    return conv


def _lattice_to_physical_wrong(kind):
    right = O.lattice_to_physical

    def conv(gamma, lam, s):
        # rescale the lattice state so that the correct readback returns
        # what the wrong power would
        if kind == "momentum":
            t = O.State(s.rho, s.mx / lam, None if s.my is None else s.my / lam,
                        s.rhoE)
        else:  # energy read back with lambda instead of lambda^2
            t = O.State(s.rho, s.mx, s.my, s.rhoE * lam)
        return right(gamma, lam, t)
    return conv


@pytest.mark.parametrize("mistake", ["pressure", "velocity", "momentum",
                                     "energy"])
def test_planted_lambda_powers_are_caught(monkeypatch, mistake):
    if mistake in ("pressure", "velocity"):
        monkeypatch.setattr(O, "prims_to_lattice",
                            _prims_to_lattice_wrong(mistake))
    else:
        monkeypatch.setattr(O, "lattice_to_physical",
                            _lattice_to_physical_wrong(mistake))
    # the conservation-law pin catches every one (toro1 carries velocity)
    assert max(totals_follow_fluxes("sod", 0.5),
               totals_follow_fluxes("toro1", 0.5)) > 1e-3
    # so does the exact-solution pin
    assert not (l1_at_half_matches("sod") and l1_at_half_matches("toro1"))
    # the lattice-unit pin sees only the forward pressure conversion (the
    # tube starts at rest and nothing is read back)
    if mistake == "pressure":
        assert lattice_momentum_growth(0.5) > 1e-3
