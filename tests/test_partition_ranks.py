"""Independent solves split across ranks (paper_1602_02675_gb300/partition):
every unit goes to exactly one rank, the work is balanced, and two gloo
ranks on the CPU end with the same results as one rank.  The solves here are
oracle runs of small tubes, standing in for the GPU batch each rank would
run: the partition logic is the same."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1602_02675_gb300 import inputs as I
from paper_1602_02675_gb300 import partition as Pt


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("count,world", [(0, 3), (1, 4), (7, 2), (100, 8),
                                         (4096, 8)])
def test_assign_covers_every_unit_once_and_balances(count, world):
    rng = np.random.default_rng(count + world)
    work = rng.uniform(1.0, 100.0, count)
    parts = Pt.assign(work, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(count))
    if count:
        loads = [sum(work[i] for i in p) for p in parts]
        # longest-first greedy: no rank exceeds the mean by more than the
        # largest unit
        assert max(loads) <= sum(work) / world + work.max() + 1e-9
    assert Pt.assign(work, world) == parts     # deterministic


def _specs():
    specs = I.tubes_batch(9, seed=44, nmin=24, nmax=64)
    out = []
    for t in specs:
        nsteps, lam = t.steps_and_lambda(0.05)
        out.append((t, nsteps, lam))
    return out


def _solve(units):
    from oracle import oracle as O
    res = {}
    for k, (t, nsteps, lam) in enumerate(units):
        P = O.Params(dim=1, nx=t.n, bc_x=O.TRANSMISSIVE)
        s, _ = O.run(P, O.riemann_planar(P, 0, 1, 0.5, t.left, t.right, lam),
                     nsteps)
        res[k] = s.rho.tolist()
    return res


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = _specs()
        work = [t.n * ns for t, ns, _ in units]
        got = Pt.solve_partitioned(units, work, _solve, rank, world,
                                   group=torch.distributed.group.WORLD)
        mine = Pt.solve_partitioned(units, work, _solve, rank, world)
        out[rank] = (got, sorted(mine))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_solve_each_unit_once_like_one_rank():
    world = 2
    units = _specs()
    work = [t.n * ns for t, ns, _ in units]
    one = Pt.solve_partitioned(units, work, _solve, 0, 1)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world,
                 join=True)
        res = dict(out)
    parts = Pt.assign(work, world)
    for rank in range(world):
        got, mine = res[rank]
        assert mine == parts[rank]            # each rank solved its share
        assert sorted(got) == list(range(len(units)))
        for k in range(len(units)):
            assert got[k] == one[k]           # same result as on one rank
    assert sorted(parts[0] + parts[1]) == list(range(len(units)))
