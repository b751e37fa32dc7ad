"""The benchmark's host-side baselines for the batched form: the oracle
sharded over spawned processes, and the operation list that replays a
batched trace through the CUDA allocators (CPU only)."""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAIL = np.uint64(0xFFFFFFFFFFFFFFFF)


def _batched_trace(n_arenas=6, n_batches=5):
    """A small batched trace driven by per-arena oracles, in the layout
    bench.py records (row offsets, host requests, results, statuses)."""
    import oracle
    from paper_2405_07079_gb300 import workloads

    A = workloads.multi_arena_sizes(n_arenas, lo=1 << 20, hi=1 << 22)
    gen = workloads.MultiLifetimes(A, n_batches=n_batches, max_ops=64, mean_life=50.0)
    ors = [oracle.Oracle(int(a), 256) for a in A]
    batches = []
    while (b := gen.next_batch()) is not None:
        frow, f, arow, s = b
        out = np.empty(s.size, np.uint64)
        st = np.empty(f.size, np.uint8)
        for i in range(n_arenas):
            o, t = ors[i].batch(f[frow[i]:frow[i + 1]], s[arow[i]:arow[i + 1]])
            out[arow[i]:arow[i + 1]] = o
            st[frow[i]:frow[i + 1]] = t
        gen.feed(out)
        batches.append({"hfrow": frow, "harow": arow, "hf": f, "hs": s, "ref_out": out, "ref_st": st})
    return A, batches


def test_oracle_pool_matches_per_arena_oracles():
    sys.path.insert(0, ROOT)
    import bench

    A, batches = _batched_trace()
    seqs = [[(b["hf"][b["hfrow"][i]:b["hfrow"][i + 1]], b["hs"][b["harow"][i]:b["harow"][i + 1]]) for b in batches]
            for i in range(len(A))]
    v, cores, res = bench.oracle_pool_baseline(A, 256, seqs, cores=2)
    assert v > 0 and cores == 2
    for i in range(len(A)):
        for bi, b in enumerate(batches):
            assert np.array_equal(res[i][bi][0], b["ref_out"][b["harow"][i]:b["harow"][i + 1]])


def test_cuda_replay_ops_multi_is_well_formed():
    sys.path.insert(0, ROOT)
    import bench

    A, batches = _batched_trace()
    ops = bench.cuda_replay_ops_multi(batches, range(len(A)))
    live, n = set(), 0
    for op in ops.tolist():
        if op >= 0:
            live.add(n); n += 1
        else:
            assert -op - 1 in live
            live.remove(-op - 1)
    assert n == sum(int((b["ref_out"] != FAIL).sum()) for b in batches)


def test_space_report_definitions():
    """The memory-usage summary: fragmentation 1 - live / extent, rounding
    1 - live / used, largest free / free bytes; batches with nothing in use
    or nothing free are left out of the ratios they would divide by zero."""
    sys.path.insert(0, ROOT)
    import bench

    samples = [(0, 0, 0, 4096, 4096),        # nothing live yet
               (50, 64, 100, 30, 40),
               (300, 400, 1000, 0, 0)]       # arena full
    r = bench.space_report(samples, 4096)
    assert r["fragmentation"]["mean"] == (0.5 + 0.7) / 2
    assert r["fragmentation"]["final"] == 0.7 and r["fragmentation"]["max"] == 0.7
    assert r["rounding"]["mean"] == ((1 - 50 / 64) + (1 - 300 / 400)) / 2
    assert r["largest_free_over_free"]["mean"] == (1.0 + 0.75) / 2
    assert r["peak_extent_bytes"] == 1000 and r["arena_bytes"] == 4096
    assert r["series"]["rows"][1] == [50, 64, 100]
