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


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def join(self, timeout=None):
        pass


def _clocks(lines):
    import bench
    c = object.__new__(bench.Clocks)
    c.proc, c.reader, c.lines = _Done(), _Done(), list(lines)
    return c.stop()


def test_clock_samples_give_median_max_and_throttle_reasons():
    """The clock record of the timed region (nvidia-smi samples of SM clock,
    its maximum and the throttle reasons): the median under load, the
    largest maximum, and every reason seen Active; malformed lines skipped."""
    ok = "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1950, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1300.0, 0x8, Not Active, Active, Not Active, Not Active"
    r = _clocks([ok, ok, cap, "garbage", ok])
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 4
    r = _clocks([ok, hot, hot])
    assert r["sm_mhz"] == 1500.0
    assert r["reasons"] == ["hw_thermal_slowdown"]
    r = _clocks([])
    assert r["sm_mhz"] is None and r["reasons"] == [] and r["samples"] == 0
