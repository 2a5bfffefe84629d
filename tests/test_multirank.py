"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1 check the
view sharding (disjoint frames per step) and the whole-job timing reduction
(max of the ranks' times, sum of their samples)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    views = [bench.rank_views(k, rank, world) for k in range(8)]
    t, n = bench.aggregate(1.0 + rank, 100 * (rank + 1), world, "cpu")
    q.put((rank, views, t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing_reduction():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict()
    for _ in range(world):
        r, views, t, n = q.get(timeout=120)
        res[r] = (views, t, n)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k in range(8):
        assert res[0][0][k] != res[1][0][k]  # the ranks render different frames each step
    assert res[0][1] == res[1][1] == 2.0  # slowest rank
    assert res[0][2] == res[1][2] == 300  # all samples
    import bench
    assert bench.aggregate(3.5, 7, 1, "cpu") == (3.5, 7)
