"""The benchmark's multi-rank aggregation (replicas: no collective on the
data path, only the final MAX of times and SUM of counts), run as two gloo
ranks on the CPU."""
from __future__ import annotations

import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: times (1 + r, 10 - r) seconds, counts (100 * (r + 1), 7)
        maxes, sums = bench.reduce_over_ranks([1.0 + rank, 10.0 - rank], [100 * (rank + 1), 7], world)
        q.put((rank, maxes, sums))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, maxes, sums in got:
        assert maxes == [2.0, 10.0]
        assert sums == [300.0, 14.0]


def test_reduce_is_identity_for_one_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks([1.5, 2], [3, 4], 1) == ([1.5, 2.0], [3.0, 4.0])
