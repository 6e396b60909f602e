"""Multi-GPU layout of the benchmark, exercised on the CPU with gloo (world
size 2): clips are sharded across ranks with no data-path collective, and the
job time is the slowest rank's (the only collective is that MAX)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.clip_seeds(1000, rank, world, clips_per_rank=2)
        local_ms = 10.0 + 5.0 * rank
        job = bench.job_time_ms(local_ms, dist, "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out[rank] = (seeds, job, gathered)
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    s0, j0, g0 = out[0]
    s1, j1, _ = out[1]
    assert s0 == [1000, 1001] and s1 == [1002, 1003]
    assert not set(g0[0]) & set(g0[1])      # disjoint clips per rank
    assert j0 == j1 == 15.0                  # both ranks report the slowest rank's time


def test_single_process_time_passthrough():
    assert bench.job_time_ms(12.5) == 12.5
    assert bench.clip_seeds(7, 0, 1) == [7]
