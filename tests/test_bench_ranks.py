"""The bench's multi-GPU form (independent replicas, one rank per GPU) on CPU: two gloo
ranks with different step times both report the slowest rank's time, and the whole-job
rate counts every rank's units over it."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms_local = [120.0, 150.0][rank]
    value, ms = bench.job_rate(torch, dist, ms_local, 1000.0, world, "cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_takes_the_slowest_rank():
    world = 2
    out = mp.get_context("spawn").Manager().dict()      # no fork of this multi-threaded process
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, ms = out[r]
        assert ms == 150.0
        assert value == pytest.approx(world * 1000.0 / 0.150)


def test_single_rank_rate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_rate(torch, None, 200.0, 500.0, 1, "cpu")
    assert ms == 200.0 and value == pytest.approx(2500.0)
