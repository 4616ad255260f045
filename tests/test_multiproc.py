"""The N > 1 path of bench.py on the CPU: two gloo ranks, each an independent replica (no data
exchange), the timed region's max over ranks and the whole-job rate."""
from __future__ import annotations

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, times, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        rate = bench.whole_job_rate(1000, 10, world, ms)
        out[rank] = (ms, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_max_and_rate():
    world = 2
    times = [3.0, 5.0]
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 5.0
        assert rate == pytest.approx(1000 * 10 * world / 5e-3)


def test_single_process_path():
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.whole_job_rate(10, 4, 1, 2.0) == pytest.approx(10 * 4 / 2e-3)
