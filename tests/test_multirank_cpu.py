"""The N > 1 path of bench.py on CPU: world_size-2 gloo process group (127.0.0.1).

Every rank propagates its own replica (independent states, no data-path collective);
the job time is the slowest rank's, taken with one all-reduce of the timings.
"""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        env = bench._dist()
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        rate = bench.job_rate(1000, 4, world, slowest)
        dist.barrier()
        q.put((rank, env, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_timing_reduction_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, slowest, rate in out:
        assert env == (rank, 2, rank)
        assert slowest == 15.0                       # the slower rank's time, on both ranks
        assert rate == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_rate(9341 * 1000, 20, 1, 3.7) == pytest.approx(9341e3 * 20 / 3.7e-3)
