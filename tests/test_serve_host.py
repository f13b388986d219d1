"""Host logic of the serving loop (paper_1602_02675_gb300/serve.py) on the
CPU: the scheduler runs against stand-ins of the library's handles and of
CUDA streams, so admission against the memory budget, waiting, batching of
the FP32 2-D grids of a round and retirement are checked without a GPU.
(The solves themselves are checked on the GPU in test_gpu_serve.py.)"""
import math

import numpy as np
import pytest

from paper_1602_02675_gb300 import lbm as L
from paper_1602_02675_gb300 import serve as S


class _Stream:
    cuda_stream = None


class _Pool:
    """Tube pool stand-in: a node budget; add raises LBM_EBUDGET when full."""

    def __init__(self, capacity_nodes, max_slots=4096, precision=L.F32,
                 stream=None):
        self.cap, self.used, self.slots = capacity_nodes, 0, {}
        self.next = 0

    def add(self, tube):
        if self.used + tube.n > self.cap:
            raise L.LbmError(L.EBUDGET, "pool full")
        self.used += tube.n
        self.next += 1
        self.slots[self.next] = tube
        return self.next

    def run(self, k):
        assert k >= 1

    def read(self, slot):
        return {"rho": np.ones(self.slots[slot].n)}

    def remove(self, slot):
        self.used -= self.slots.pop(slot).n

    def close(self):
        pass


class _Solver:
    live = 0

    def __init__(self, cfg):
        self.n = cfg.nx * cfg.ny
        _Solver.live += 1

    def init_riemann(self, *a):
        pass

    def step(self, n):
        assert n >= 1

    def moments(self):
        return {"rho": np.ones(self.n)}

    def close(self):
        _Solver.live -= 1


class _Batch2D:
    live = 0

    def __init__(self, grids, stream=None):
        self.n = [g.cfg.nx * g.cfg.ny for g in grids]
        _Batch2D.live += 1

    def run(self, k):
        assert k >= 1

    def moments(self, i):
        return {"rho": np.ones(self.n[i])}

    def close(self):
        _Batch2D.live -= 1


@pytest.fixture
def fakes(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "Stream", _Stream)
    monkeypatch.setattr(S.L, "Pool", _Pool)
    monkeypatch.setattr(S.L, "Solver", _Solver)
    monkeypatch.setattr(S.L, "Batch2D", _Batch2D)
    _Solver.live = _Batch2D.live = 0
    yield


@pytest.mark.parametrize("precision", [L.F32, L.F64])
def test_every_request_is_served_once_within_the_budget(fakes, precision):
    reqs = S.mixed_requests(120, seed=3, n1=(512, 8192), n2=(64, 512))
    budget = 256 << 20   # the largest FP64 grid here needs ~95 MB
    srv = S.Server(budget=budget, precision=precision, pool_nodes=1 << 16,
                   steps_per_tick=50)
    for r in reqs:
        srv.submit(r, now=0.0)
    srv.drain()
    assert not srv.busy()
    assert len(srv.results) + len(srv.errors) == len(reqs)
    assert not srv.errors
    assert srv.peak_used <= budget
    for r in reqs:
        res = srv.results[r.rid]
        assert res.steps == r.steps_and_lambda()[0]
        assert res.fields["rho"].size == r.nodes()
    # every handle was released
    assert _Solver.live == 0 and _Batch2D.live == 0
    assert srv._pool.used == 0


def test_requests_too_large_are_rejected_and_the_rest_wait(fakes):
    big = S.Request(0, 2, 4096, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.1,
                    ny=4096)
    small = [S.Request(i, 2, 256, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.05,
                       ny=256) for i in range(1, 9)]
    need = S.bytes_needed(small[0], L.F64)
    pool_bytes = (1 << 10) * 2 * 3 * 8
    # room for two of the small grids at a time
    srv = S.Server(budget=pool_bytes + 2 * need + need // 2,
                   precision=L.F64, pool_nodes=1 << 10, steps_per_tick=4)
    for r in [big] + small:
        srv.submit(r, now=0.0)
    srv.tick()
    assert "EBUDGET" in srv.errors[0]
    assert len(srv._a2) == 2 and len(srv.pending) == 6
    srv.drain()
    assert sorted(srv.results) == list(range(1, 9))
    assert srv.peak_used <= srv.budget


def test_steps_and_lambda_reach_t_end_within_the_speed_limit():
    """Whole steps to t_end with lambda = dt/dx <= 1 and lambda^2 max(p/rho)
    <= 1 (the hot-tube reading of the units)."""
    for right in ((0.125, 0.0, 0.1), (0.5, 0.0, 3.0), (0.1, 0.0, 9.0)):
        r = S.Request(0, 1, 1000, (1.0, 0.0, 1.0), right, 0.2)
        steps, lam = r.steps_and_lambda()
        hot = max(1.0, right[2] / right[0])
        assert lam <= 1.0 and lam * lam * hot <= 1.0 + 1e-12
        assert math.isclose(steps * lam / r.n, 0.2, rel_tol=1e-13)
        # the next smaller step count would exceed the limit
        assert 0.2 / ((steps - 1) / r.n) > 1.0 / math.sqrt(hot) - 1e-12


def test_request_mix_and_arrivals():
    reqs = S.mixed_requests(2000, seed=11)
    d1 = [r for r in reqs if r.dim == 1]
    assert 0.65 < len(d1) / len(reqs) < 0.75
    assert all(512 <= r.n <= 65536 for r in d1)
    assert all(256 <= r.n <= 2048 and r.ny == r.n for r in reqs if r.dim == 2)
    assert all(0.05 <= r.t_end <= 0.25 for r in reqs)
    again = S.mixed_requests(2000, seed=11)
    assert [(r.dim, r.n, r.t_end) for r in again] == \
        [(r.dim, r.n, r.t_end) for r in reqs]
    t = S.poisson_arrivals(5000, rate=50.0, seed=2)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 50.0) < 0.002
