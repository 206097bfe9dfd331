"""The bench's multi-rank host logic on CPU: two gloo ranks (127.0.0.1).

Under torchrun each rank solves its own seeded instance; the timed region is
bracketed by barriers, the time is the maximum over ranks and the value is
the units all ranks processed divided by it (weak scaling).  The reference arm
runs on rank 0 only; other ranks return at once.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    import bench
    import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                      # this rank's timed region
        bench.barrier(world)
        mx = bench.max_over_ranks(ms, world, "cpu")
        thr = bench.job_throughput(3, world, mx / 1e3)
        seed = bench.rank_seed(rank)
        _, _, ph = W.one_ellipse_640(seed=seed)
        ref = None
        if rank != 0:
            class A:
                steps, warmup, gpus = 2, 1, world
            ref = bench.run_reference(A())
        q.put((rank, mx, thr, seed, float(ph.sum()), ref))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, thr0, s0, ph0, _), (r1, mx1, thr1, s1, ph1, ref1) = res
    assert mx0 == mx1 == 15.0                      # the slowest rank's time, on every rank
    assert thr0 == thr1 == pytest.approx(2 * 3 / 0.015)
    assert s0 != s1 and ph0 != ph1                 # each rank its own instance
    assert ref1 == 0                               # reference arm: rank 1 does no work
