"""The multi-rank reporting of bench.py (one independent restoration per rank,
weak scaling) on two gloo ranks on the CPU: the job's time is the slowest
rank's, and throughput counts every rank's work."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, rank, world)
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        t = bench.max_over_ranks(ms, world, torch.device("cpu"))
        v = bench.replica_throughput(1024 * 1024, 50, 4, world, t)
        dist.barrier()
        out[rank] = (t, v)
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_is_the_slowest_rank_and_counts_all_work():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == pytest.approx(15.0)
        assert v == pytest.approx(1024 * 1024 * 50 * 4 * 2 / 1e6 / 0.015)


def test_single_rank_is_the_identity():
    import bench

    assert bench.max_over_ranks(12.5, 1, torch.device("cpu")) == 12.5
    assert bench.replica_throughput(100, 10, 2, 1, 1000.0) == pytest.approx(100 * 10 * 2 / 1e6)
