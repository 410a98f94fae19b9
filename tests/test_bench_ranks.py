"""The replica path of bench.py (--gpus N > 1) on CPU: two gloo ranks, each
with its own step time; the whole-job rate uses the slowest rank's time and
every rank agrees on it."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (ms_max, bench.whole_job_rate(world, 3, ms_max / 1e3))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_max, rate = res[0]
    assert ms_max == 150.0
    assert abs(rate - 2 * 3 / 0.150) < 1e-9


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5, None, "cpu") == 42.5
    assert bench.whole_job_rate(1, 3, 1.5) == 2.0
