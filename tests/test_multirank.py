"""World-size-2 gloo test of the benchmark's multi-rank protocol on CPU:
barrier-bracketed timing, max over ranks, whole-job throughput and the
per-rank trajectory seeds (weak scaling, no data-path collective)."""
import os
import socket
import sys
import time

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    delay = 0.05 * (rank + 1)
    t = bench.timed_region(lambda: time.sleep(delay), world)
    v = bench.job_throughput(10, world, t)
    seed = bench.rank_trajectory_seed(7, rank, world)
    q.put((rank, t, v, seed))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_protocol():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, v0, s0), (_, t1, v1, s1) = res
    assert t0 == t1 and t0 >= 0.1            # both ranks see the slowest rank's time
    assert abs(v0 - 20 / t0) < 1e-9 and v0 == v1
    assert s0 != s1                           # each rank renders its own trajectory


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_trajectory_seed(3, 0, 1) == 3
    assert bench.job_throughput(30, 1, 0.5) == 60.0
    assert bench.max_over_ranks(1.5, 1) == 1.5
