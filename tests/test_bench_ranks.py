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


def _bench(args, rank, world):
    import subprocess

    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], env=env, cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_on_rank_zero_only():
    """`bench.py --impl reference` as two ranks of one job: rank 0 prints one
    JSON line with the contract's keys, the other rank exits 0 silently."""
    import json

    args = ["--impl", "reference", "--workload", "tiny", "--steps", "20", "--warmup", "3"]
    r1 = _bench(args, 1, 2)
    assert r1.returncode == 0 and r1.stdout.strip() == "", r1.stderr[-2000:]
    r0 = _bench(args, 0, 2)
    assert r0.returncode == 0, r0.stderr[-2000:]
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 20
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_of_every_policy():
    """The reference arm runs the oracle of each policy."""
    import json

    for policy, workload in (("tlsf", "tiny"), ("first", "usage"), ("bitmask", "objects")):
        r = _bench(["--impl", "reference", "--workload", workload, "--policy", policy, "--steps", "10",
                    "--warmup", "3"], 0, 1)
        assert r.returncode == 0, r.stderr[-2000:]
        d = json.loads(r.stdout.strip().splitlines()[-1])
        assert d["config"]["policy"] == policy and d["value"] > 0
