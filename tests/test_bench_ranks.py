"""The multi-process path of bench.py on CPU: two gloo ranks, each timing its own
replica, agree on the slowest rank's time and on the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (ms, bench.whole_job_value(3, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_value():
    world = 2
    times = [1200.0, 1500.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 1500.0
        assert value == pytest.approx(3 * world / 1.5)


def test_single_process_keeps_its_time():
    import bench
    assert bench.max_over_ranks(123.0, None, "cpu") == 123.0
    assert bench.whole_job_value(2, 1, 500.0) == pytest.approx(4.0)
