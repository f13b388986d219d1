"""Brute force: the FP64 oracle against the exact rational tracer on lattices
of 16 nodes or fewer, a few steps, every boundary kind."""
import itertools
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import oracle as O
from tests import brute_rational as B

GAMMA = F(7, 5)
THETA = F(1, 2)


def _dyadic_state(dim, shape, seed):
    """Random states whose moments are exact in binary (dyadic rationals), so
    the FP64 oracle and the tracer start from the same numbers."""
    rng = np.random.default_rng(seed)
    st = {}
    nodes = itertools.product(*[range(n) for n in shape]) if dim == 2 else \
        ((x,) for x in range(shape[0]))
    for nd in nodes:
        nd = tuple(nd)
        rho = F(int(rng.integers(4, 64)), 16)
        V = [F(int(rng.integers(-96, 97)), 64) for _ in range(dim)]
        e = F(int(rng.integers(8, 256)), 64)
        m = tuple(rho * v for v in V)
        rhoE = rho * (e + sum(v * v for v in V) / 2)
        # round m and rhoE to dyadics: keep exact binary values
        m = tuple(F(round(mi * 4096), 4096) for mi in m)
        rhoE = F(round(rhoE * 4096), 4096)
        st[nd] = (rho, m, rhoE)
    return st


def _to_oracle(dim, shape, st):
    nx = shape[0]
    ny = shape[1] if dim == 2 else 1
    N = nx * ny
    rho, mx, my, E = (np.zeros(N) for _ in range(4))
    for nd, (r, m, e) in st.items():
        i = nd[0] + (nd[1] * nx if dim == 2 else 0)
        rho[i], mx[i], E[i] = float(r), float(m[0]), float(e)
        if dim == 2:
            my[i] = float(m[1])
    return O.State(rho, mx, my if dim == 2 else None, E)


def _compare(dim, shape, exact, s):
    nx = shape[0]
    fields = [("rho", s.rho, lambda v: v[0]), ("mx", s.mx, lambda v: v[1][0]),
              ("rhoE", s.rhoE, lambda v: v[2])]
    if dim == 2:
        fields.append(("my", s.my, lambda v: v[1][1]))
    for name, arr, get in fields:
        ref = np.zeros_like(arr)
        for nd, v in exact.items():
            ref[nd[0] + (nd[1] * nx if dim == 2 else 0)] = float(get(v))
        scale = np.max(np.abs(ref))
        err = np.max(np.abs(arr - ref))
        assert err <= 1e-14 * scale, (name, err / scale)


CASES_1D = [
    (O.PERIODIC, 12, 3), (O.PERIODIC, 16, 2), (O.TRANSMISSIVE, 14, 3),
    (O.REFLECTING, 16, 3),
]


@pytest.mark.parametrize("bc,n,steps", CASES_1D)
def test_oracle_matches_exact_tracer_1d(bc, n, steps):
    st = _dyadic_state(1, (n,), seed=100 + n + bc)
    P = O.Params(dim=1, nx=n, gamma=1.4, theta=0.5, bc_x=bc)
    s = _to_oracle(1, (n,), st)
    exact = st
    for _ in range(steps):
        exact = B.step(1, (n,), (bc,), GAMMA, THETA, exact)
        s, _, _ = O.step(P, s)
        _compare(1, (n,), exact, s)


CASES_2D = [
    ((O.PERIODIC, O.PERIODIC), (4, 4), 2),
    ((O.TRANSMISSIVE, O.REFLECTING), (4, 3), 2),
    ((O.REFLECTING, O.PERIODIC), (3, 5), 1),
    ((O.TRANSMISSIVE, O.TRANSMISSIVE), (3, 3), 1),
]


@pytest.mark.parametrize("bcs,shape,steps", CASES_2D)
def test_oracle_matches_exact_tracer_2d(bcs, shape, steps):
    st = _dyadic_state(2, shape, seed=200 + shape[0] * 7 + shape[1] + bcs[0])
    P = O.Params(dim=2, nx=shape[0], ny=shape[1], gamma=1.4, bc_x=bcs[0],
                 bc_y=bcs[1])
    s = _to_oracle(2, shape, st)
    exact = st
    for _ in range(steps):
        exact = B.step(2, shape, bcs, GAMMA, THETA, exact)
        s, _, _ = O.step(P, s)
        _compare(2, shape, exact, s)
