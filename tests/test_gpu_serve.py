"""Continuous-batching server: every result is the same served alone and
in the mix, 1-D results match the FP64 oracle, the memory budget holds."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1602_02675_gb300 import lbm as L
from paper_1602_02675_gb300 import serve as S

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "mx", "rhoE", "p")


def _mix():
    return S.mixed_requests(14, seed=31, n1=(200, 3000), n2=(48, 160),
                            t_range=(0.05, 0.15))


@pytest.mark.parametrize("precision", [L.F32, L.F64])
def test_results_same_alone_and_in_the_mix(precision):
    reqs = _mix()
    srv = S.Server(budget=8 << 30, precision=precision, pool_nodes=1 << 18,
                   max_slots=64)
    try:
        arrivals = np.linspace(0.0, 0.05, len(reqs))
        stats = S.run_trace(srv, reqs, arrivals)
        assert stats["solves"] == len(reqs) and stats["errors"] == 0
        mixed = {k: v.fields for k, v in srv.results.items()}
    finally:
        srv.close()
    assert {r.dim for r in reqs} == {1, 2}
    for r in reqs:
        one = S.Server(budget=8 << 30, precision=precision, pool_nodes=1 << 18,
                       max_slots=4)
        try:
            q = S.Request(r.rid, r.dim, r.n, r.left, r.right, r.t_end, ny=r.ny)
            one.submit(q)
            one.drain()
            alone = one.results[r.rid].fields
        finally:
            one.close()
        for f in FIELDS:
            assert np.array_equal(alone[f], mixed[r.rid][f]), (r.rid, r.dim, f)


def test_served_tubes_match_oracle():
    reqs = [r for r in _mix() if r.dim == 1]
    srv = S.Server(budget=8 << 30, precision=L.F64, pool_nodes=1 << 18,
                   max_slots=64)
    try:
        for r in reqs:
            srv.submit(r)
        srv.drain()
        for r in reqs:
            steps, lam = r.steps_and_lambda()
            lam = (lam / r.n) * r.n     # the library forms dt * n
            P = O.Params(dim=1, nx=r.n, bc_x=O.TRANSMISSIVE)
            st, _ = O.run(P, O.riemann_planar(P, 0, 1, r.x_d, r.left, r.right,
                                             lam), steps)
            o = O.lattice_to_physical(1.4, lam, st)
            g = srv.results[r.rid].fields
            for f in ("rho", "mx", "rhoE"):
                assert np.array_equal(g[f], o[f]), (r.rid, f)
    finally:
        srv.close()


def test_budget_is_respected_and_oversize_rejected():
    reqs = [r for r in _mix() if r.dim == 2]
    big = max(S.bytes_needed(r, L.F32) for r in reqs)
    pool_nodes = 1 << 12
    budget = pool_nodes * 24 + big + big // 2   # room for about one grid
    srv = S.Server(budget=budget, precision=L.F32, pool_nodes=pool_nodes,
                   max_slots=8)
    try:
        huge = S.Request(999, 2, 4096, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1),
                         0.1, ny=4096)
        for r in reqs + [huge]:
            srv.submit(r)
        srv.drain()
        assert srv.peak_used <= budget
        assert 999 in srv.errors and "EBUDGET" in srv.errors[999]
        assert set(srv.results) == {r.rid for r in reqs}
    finally:
        srv.close()


def _oracle_request(r, fp32_storage=False):
    """The oracle's run of a served request (physical units), optionally
    with its state rounded to FP32 after every step (the floor any FP32
    path can reach where the flow amplifies rounding)."""
    steps, lam = r.steps_and_lambda()
    # the lambda the library forms from dt = lam / n: the pool dt * n, a
    # handle dt / dx with dx = 1 / n
    lam = (lam / r.n) * r.n if r.dim == 1 else (lam / r.n) / (1.0 / r.n)
    if r.dim == 1:
        P = O.Params(dim=1, nx=r.n, bc_x=O.TRANSMISSIVE)
        left, right = r.left, r.right
    else:
        P = O.Params(dim=2, nx=r.n, ny=r.ny, bc_x=O.TRANSMISSIVE,
                     bc_y=O.REFLECTING)
        left = (r.left[0], r.left[1], 0.0, r.left[2])
        right = (r.right[0], r.right[1], 0.0, r.right[2])
    st = O.riemann_planar(P, 0, 1, r.x_d, left, right, lam)
    if not fp32_storage:
        st, _ = O.run(P, st, steps)
    else:
        q = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)
        st = O.State(q(st.rho), q(st.mx), q(st.my), q(st.rhoE))
        for _ in range(steps):
            st, _, _ = O.step(P, st)
            st = O.State(q(st.rho), q(st.mx), q(st.my), q(st.rhoE))
    return O.lattice_to_physical(1.4, lam, st)


def test_served_2d_grids_fp64_match_oracle():
    """2-D grids served in the mix, FP64: bit for bit with the oracle."""
    reqs = _mix()
    srv = S.Server(budget=8 << 30, precision=L.F64, pool_nodes=1 << 18,
                   max_slots=64)
    try:
        S.run_trace(srv, reqs, np.linspace(0.0, 0.05, len(reqs)))
        grids = [r for r in reqs if r.dim == 2]
        assert grids
        for r in grids:
            o = _oracle_request(r)
            g = srv.results[r.rid].fields
            for f in ("rho", "mx", "rhoE"):
                assert np.array_equal(g[f], o[f]), (r.rid, f)
    finally:
        srv.close()


def test_served_fp32_match_oracle():
    """Every request of the mix served in FP32 (1-D tubes in the pool, 2-D
    grids on the deposit kernel) against the FP64 oracle: mean |error| at
    most 1e-5 of each field's range, or within 4x of what the oracle itself
    loses by rounding its state to FP32 every step where the flow amplifies
    rounding."""
    reqs = _mix()
    srv = S.Server(budget=8 << 30, precision=L.F32, pool_nodes=1 << 18,
                   max_slots=64)
    try:
        S.run_trace(srv, reqs, np.linspace(0.0, 0.05, len(reqs)))
        for r in reqs:
            o = _oracle_request(r)
            g = srv.results[r.rid].fields
            floor = None
            for f in ("rho", "mx", "rhoE"):
                rng = o[f].max() - o[f].min()
                err = np.mean(np.abs(g[f] - o[f])) / rng
                if err > 1e-5:
                    if floor is None:
                        floor = _oracle_request(r, fp32_storage=True)
                    ferr = np.mean(np.abs(floor[f] - o[f])) / rng
                    assert err <= 4.0 * ferr, (r.rid, r.dim, f, err, ferr)
    finally:
        srv.close()
