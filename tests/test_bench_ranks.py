"""The multi-rank path of the benchmark (independent replicas, max-over-ranks
timing, whole-job rate) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 10.0 - rank]       # ranks finish at different times
        got = bench.max_over_ranks(mine, world, "cpu")
        out[rank] = (got, bench.job_rate(1000, world, got[0]))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world,
                 join=True)
        res = dict(out)
    for rank in range(world):
        got, rate = res[rank]
        assert got == [2.0, 10.0]
        assert rate == pytest.approx(2 * 1000 / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.job_rate(10, 1, 2.0) == 5.0
