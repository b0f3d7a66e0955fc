"""The multi-GPU path of the benchmark runs independent replicas (the
reductions shard without any data-path exchange): each rank times its own
replica between barriers and the job's step time is the maximum over ranks.
These CPU tests run that host logic with the gloo backend at world size 2."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, step_ms, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(step_ms[rank], dist, torch.device("cpu"))
        out[rank] = (slowest, bench.job_throughput(1000, world, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_max_over_ranks_and_value_sums_replicas():
    world = 2
    step_ms = [120.0, 150.0]
    with mp.get_context("spawn").Manager() as m:  # no fork of this (multi-threaded) process
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), step_ms, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        slowest, value = res[r]
        assert slowest == 150.0
        assert value == pytest.approx(2 * 1000 / 0.150)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.job_throughput(300, 1, 1000.0) == pytest.approx(300.0)
