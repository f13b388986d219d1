"""Continuous-batching server for shock-tube solves.

Requests (1-D tubes or 2-D square-lattice grids with a planar Riemann jump,
Section V.C) arrive over time.  Every tick the server

1. admits waiting requests in arrival order while the device-memory budget
   has room for them (a request that does not fit waits; later, smaller
   ones may pass it);
2. advances every admitted solve by up to ``steps_per_tick`` steps: all 1-D
   tubes together with one ``lbm_pool_run`` call (a launch per step); the
   FP32 2-D grids admitted in the same round together as one batch
   (``lbm_batch2d_run``: two launches per lattice step for the whole
   batch), each batch and each FP64 grid (``lbm_step``) on its own CUDA
   stream, so their kernels overlap on the device;
3. retires the solves that reached their step count, reading their moments
   back and freeing their memory.

This module only schedules: every step of every solve runs in the CUDA
library (``liblbm.so``).  A solve's result does not depend on what else is
being served: the pool gives each tube its own step counter, and a
batched grid's steps are those of a handle of its own (bit for bit).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import lbm as L


@dataclass
class Request:
    rid: int
    dim: int               # 1 or 2
    n: int                 # nodes along x (2-D: the grid is n x ny)
    left: tuple            # (rho, u, p)
    right: tuple
    t_end: float
    ny: int = 1
    arrival: float = 0.0   # seconds, set on submit
    x_d: float = 0.5

    def steps_and_lambda(self):
        """dt/dx = 1, or scaled down for a state hotter than the Sod left
        state (lambda0^2 max(p/rho) = 1); whole steps to t_end."""
        t = max(self.left[2] / self.left[0], self.right[2] / self.right[0])
        lam0 = min(1.0, (1.0 / t) ** 0.5)
        dx = 1.0 / self.n
        steps = max(1, int(math.ceil(self.t_end / (lam0 * dx) - 1e-9)))
        return steps, self.t_end / (steps * dx)

    def nodes(self) -> int:
        return self.n * (self.ny if self.dim == 2 else 1)


def bytes_needed(req: Request, precision: int) -> int:
    """Device bytes a solve holds while admitted: 2-D grids two moment sets
    (4 fields), in FP64 one set of 248-byte source records over the grid
    padded by the reach limit 6, the FP64 readback staging (5 fields) and
    per-tile partials; 1-D tubes two sets of 3 fields in the pool."""
    b = 8 if precision == L.F64 else 4
    n = req.nodes()
    if req.dim == 2:
        rec = (0 if precision == L.F32
               else 248 * (req.n + 12) * (req.ny + 12))
        return n * (2 * 4 * b + 5 * 8) + rec + (n // 256 + 1) * 32 + (1 << 20)
    return n * 2 * 3 * b


@dataclass
class Result:
    rid: int
    fields: dict
    arrival: float
    done: float
    steps: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Active2D:
    req: Request
    solver: object       # its handle (FP64), or None when batched
    stream: object
    steps: int
    taken: int = 0
    group: object = None  # _Group2D of a batched grid
    index: int = 0        # its grid index in the batch
    done: bool = False


@dataclass
class _Group2D:
    """FP32 2-D grids admitted in one round, stepped as one batch; its
    memory is released when the last of its grids is retired."""
    batch: object
    stream: object
    live: int
    nbytes: int
    steps_done: int = 0


@dataclass
class _Active1D:
    req: Request
    slot: int
    steps: int
    taken: int = 0   # host count: every pool step advances every tube


@dataclass
class Server:
    """Continuous batching within a device-memory budget (bytes)."""
    budget: int
    precision: int = L.F32
    pool_nodes: int = 1 << 25
    max_slots: int = 4096
    steps_per_tick: int = 8   # steps per solve between admissions
    clock: object = time.perf_counter
    pending: list = field(default_factory=list)
    results: dict = field(default_factory=dict)
    errors: dict = field(default_factory=dict)

    def __post_init__(self):
        import torch
        self._torch = torch
        self._stream = torch.cuda.Stream()
        self._pool = L.Pool(self.pool_nodes, self.max_slots,
                            precision=self.precision,
                            stream=self._stream.cuda_stream)
        pb = 8 if self.precision == L.F64 else 4
        self._pool_bytes = self.pool_nodes * 2 * 3 * pb
        self._used = self._pool_bytes       # the pool is always resident
        self._a1: list[_Active1D] = []
        self._a2: list[_Active2D] = []
        self._spare_streams = []
        self.ticks = 0
        self.peak_used = self._used

    # ---- requests -------------------------------------------------------
    def submit(self, req: Request, now: float | None = None) -> None:
        req.arrival = self.clock() if now is None else now
        self.pending.append(req)

    def busy(self) -> bool:
        return bool(self.pending or self._a1 or self._a2)

    # ---- one scheduling round ------------------------------------------
    def tick(self) -> None:
        self._admit()
        self._advance()
        self._retire()
        self.ticks += 1

    def _admit(self) -> None:
        waiting = []
        new2d = []
        for req in self.pending:
            steps, lam = req.steps_and_lambda()
            never = (req.nodes() > self.pool_nodes if req.dim == 1 else
                     bytes_needed(req, self.precision) > self.budget - self._pool_bytes)
            if never:
                self.errors[req.rid] = "LBM_EBUDGET: larger than the budget"
                continue
            try:
                if req.dim == 1:
                    tube = L.make_tube(req.n, steps, lam / req.n, req.left,
                                       req.right, x_d=req.x_d)
                    slot = self._pool.add(tube)   # LBM_EBUDGET if full
                    self._a1.append(_Active1D(req, slot, steps))
                    continue
                need = bytes_needed(req, self.precision)
                if self._used + need > self.budget:
                    waiting.append(req)
                    continue
                if self.precision == L.F32:
                    # stepped with the others of this round as one batch
                    cfg = L.make_config(2, req.n, req.ny, dt=lam / req.n,
                                        precision=self.precision,
                                        bc_x=L.TRANSMISSIVE,
                                        bc_y=L.REFLECTING, kahan=0)
                    new2d.append((req, cfg, steps, need))
                    self._used += need
                    self.peak_used = max(self.peak_used, self._used)
                    continue
                stream = (self._spare_streams.pop() if self._spare_streams
                          else self._torch.cuda.Stream())
                cfg = L.make_config(2, req.n, req.ny, dt=lam / req.n,
                                    precision=self.precision,
                                    bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING,
                                    kahan=0, stream=stream.cuda_stream)
                s = L.Solver(cfg)
                s.init_riemann(req.left, req.right, L.PLANAR_X, req.x_d)
                self._used += need
                self.peak_used = max(self.peak_used, self._used)
                self._a2.append(_Active2D(req, s, stream, steps))
            except L.LbmError as e:
                if e.status == L.EBUDGET:
                    waiting.append(req)
                else:
                    self.errors[req.rid] = str(e)
        self.pending = waiting
        if new2d:
            stream = (self._spare_streams.pop() if self._spare_streams
                      else self._torch.cuda.Stream())
            grids = [L.make_grid2d(cfg, req.left, req.right, L.PLANAR_X,
                                   req.x_d, 0.5, 0.0, steps)
                     for req, cfg, steps, _ in new2d]
            try:
                batch = L.Batch2D(grids, stream=stream.cuda_stream)
            except L.LbmError as e:
                for req, _, _, need in new2d:
                    self.errors[req.rid] = str(e)
                    self._used -= need
                self._spare_streams.append(stream)
                return
            group = _Group2D(batch, stream, len(new2d),
                             sum(need for *_, need in new2d))
            for j, (req, _, steps, _) in enumerate(new2d):
                self._a2.append(_Active2D(req, None, stream, steps,
                                          group=group, index=j))

    def _advance(self) -> None:
        k = max(1, int(self.steps_per_tick))
        if self._a1:
            # the pool advances only the tubes still short of their steps
            kk = min(k, max(a.steps - a.taken for a in self._a1))
            self._pool.run(kk)
            for a in self._a1:
                a.taken = min(a.steps, a.taken + kk)
        groups = {}
        for a in self._a2:
            if a.group is not None:
                groups[id(a.group)] = a.group
                continue
            n = min(k, a.steps - a.taken)
            if n > 0:
                a.solver.step(n)
                a.taken += n
        for g in groups.values():
            g.batch.run(k)            # grids past their steps stay as they are
            g.steps_done += k
        for a in self._a2:
            if a.group is not None:
                a.taken = min(a.steps, a.group.steps_done)

    def _retire(self) -> None:
        keep1 = []
        for a in self._a1:
            if a.taken < a.steps:
                keep1.append(a)
                continue
            try:
                f = self._pool.read(a.slot)
                self.results[a.req.rid] = Result(a.req.rid, f, a.req.arrival,
                                                 self.clock(), a.steps)
            except L.LbmError as e:
                self.errors[a.req.rid] = str(e)
            self._pool.remove(a.slot)
        self._a1 = keep1
        keep2 = []
        for a in self._a2:
            if a.taken < a.steps:
                keep2.append(a)
                continue
            try:
                f = (a.solver.moments() if a.group is None
                     else a.group.batch.moments(a.index))
                self.results[a.req.rid] = Result(a.req.rid, f, a.req.arrival,
                                                 self.clock(), a.steps)
            except L.LbmError as e:
                self.errors[a.req.rid] = str(e)
            if a.group is None:
                a.solver.close()
                self._spare_streams.append(a.stream)
                self._used -= bytes_needed(a.req, self.precision)
                continue
            a.group.live -= 1
            if a.group.live == 0:
                a.group.batch.close()
                self._spare_streams.append(a.group.stream)
                self._used -= a.group.nbytes
        self._a2 = keep2

    def drain(self) -> None:
        while self.busy():
            self.tick()

    def close(self) -> None:
        for a in self._a2:
            if a.group is None:
                a.solver.close()
            else:
                a.group.batch.close()
        self._a2 = []
        self._a1 = []
        if getattr(self, "_pool", None) is not None:
            self._pool.close()
            self._pool = None


def solve_alone(req: Request, precision: int) -> dict:
    """The same solve through one handle, nothing else on the device (the
    plain one-solve-at-a-time path)."""
    steps, lam = req.steps_and_lambda()
    if req.dim == 1:
        cfg = L.make_config(1, req.n, dt=lam / req.n, precision=precision,
                            bc_x=L.TRANSMISSIVE)
    else:
        cfg = L.make_config(2, req.n, req.ny, dt=lam / req.n,
                            precision=precision, bc_x=L.TRANSMISSIVE,
                            bc_y=L.REFLECTING, kahan=0)
    with L.Solver(cfg) as s:
        s.init_riemann(req.left, req.right, L.PLANAR_X, req.x_d)
        s.step(steps)
        return s.moments()


def mixed_requests(count: int, seed: int, n1=(512, 65536), n2=(256, 2048),
                   frac_1d: float = 0.7, t_range=(0.05, 0.25), ny2: int = 0):
    """Seeded mix: 70 % 1-D tubes with log-uniform node counts, 30 % 2-D
    square grids with log-uniform side (ny2 > 0: fixed grid height), left
    state (1, 0, 1), right state with pressure ratio log-uniform in [2, 100]
    and density ratio uniform in [1, 10], end time uniform in t_range."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dim = 1 if rng.uniform() < frac_1d else 2
        lo, hi = n1 if dim == 1 else n2
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        pr = math.exp(rng.uniform(math.log(2.0), math.log(100.0)))
        dr = rng.uniform(1.0, 10.0)
        t_end = rng.uniform(*t_range)
        out.append(Request(i, dim, n, (1.0, 0.0, 1.0), (1.0 / dr, 0.0, 1.0 / pr),
                           t_end, ny=(ny2 or n) if dim == 2 else 1))
    return out


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))


def run_trace(server: Server, reqs, arrivals) -> dict:
    """Feed requests at their arrival times (wall clock), tick until all are
    served; returns throughput and latency percentiles."""
    t0 = server.clock()
    i = 0
    while i < len(reqs) or server.busy():
        now = server.clock() - t0
        while i < len(reqs) and arrivals[i] <= now:
            server.submit(reqs[i], t0 + arrivals[i])
            i += 1
        if server.busy():
            server.tick()
        elif i < len(reqs):
            time.sleep(max(0.0, min(0.01, arrivals[i] - now)))
    wall = server.clock() - t0
    lat = np.array([r.latency for r in server.results.values()])
    return {"solves": len(server.results), "errors": len(server.errors),
            "wall_s": wall, "solves_per_s": len(server.results) / wall,
            "latency_ms_p50": float(1e3 * np.percentile(lat, 50)) if len(lat) else None,
            "latency_ms_p99": float(1e3 * np.percentile(lat, 99)) if len(lat) else None,
            "ticks": server.ticks}
