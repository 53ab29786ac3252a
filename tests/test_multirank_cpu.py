"""The N-GPU path's host logic on CPU ranks (gloo, world size 2): each rank simulates its
own frame (replicas, no data-path collective); the only exchange is the max-over-ranks time
that turns per-rank work into the whole-job rate."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import scenegen


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 0.5 * (rank + 1)                       # rank 1 is the slow one
        slowest = bench.max_over_ranks(seconds, world, dist, "cpu")
        rate = bench.whole_job_rate(1_000, 10, world, slowest)
        _, rays = scenegen.automotive_scene(seed=bench.replica_seed(rank), n_rays=500)
        q.put((rank, slowest, rate, float(rays.range_rt_m.sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_run_distinct_frames():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, r0, f0), (_, s1, r1, f1) = out
    assert s0 == s1 == 1.0                               # both ranks see the slowest time
    assert r0 == r1 == 1_000 * 10 * 2 / 1.0              # all ranks' work over that time
    assert f0 != f1                                      # replicas simulate different frames


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(2.5, 1, None, "cpu") == 2.5
    assert bench.whole_job_rate(7, 3, 1, 2.0) == 10.5
