"""Multi-rank (replicas) host logic of bench.py on CPU with the gloo backend.

The method does not shard within a tensor, so N GPUs run N independent
replicas; what crosses ranks is only the timing: a barrier around the timed
region and the maximum step time over ranks.  These tests run two ranks as
processes on 127.0.0.1."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    ms = bench.max_over_ranks(1.5 + rank, world)
    value = bench.replica_value(1e9, ms, world)
    # the reference arm does its work on rank 0 only; other ranks return at once
    class A:
        nnz, warmup, steps = 1000, 0, 1
    if rank != 0:
        bench.run_reference(A, rank, world)
    bench.barrier(world)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_value():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 2.5                      # the slowest rank's time on every rank
        assert abs(value - 2 * 1e9 / 2.5e-3 / 1e9) < 1e-9
