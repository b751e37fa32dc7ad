"""GPU path vs the CPU oracle, bit-exact on every offset, every free status,
the counters and the final canonical state (all integer work)."""
from __future__ import annotations

import numpy as np
import pytest

from _helpers import FAIL, canary_intact, check_invariants, first_diff, from_dev, oracle_trace, to_dev

pytestmark = pytest.mark.gpu

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30


def _run(wl, threads=None, max_batches=None, state_every=0, canary=False, ctas=0, policy="segfit"):
    import torch

    from paper_2405_07079_gb300 import Allocator

    import oracle

    dev = torch.device("cuda")
    trace, o = oracle_trace(wl, max_batches, policy)
    lock = oracle.Oracle(wl.arena, wl.min_block, policy) if state_every else None  # replayed in lock step
    guard = None
    if canary:
        # a real arena of the managed size, filled with the canary byte; the
        # allocator never receives its address, so it must stay untouched
        guard = torch.full((wl.arena,), 0xA5, dtype=torch.uint8, device=dev)
    with Allocator(wl.arena, wl.min_block, threads=threads, ctas=ctas, policy=policy) as a:
        for b, (f, s, out, st) in enumerate(trace):
            dst = torch.empty(f.size, dtype=torch.uint8, device=dev)
            go = from_dev(a.step(to_dev(f, dev), to_dev(s, dev), status=dst)) if s.size else np.zeros(0, np.uint64)
            if not s.size:
                a.step(to_dev(f, dev), None, status=dst)
            i = first_diff(go, out)
            assert i is None, f"batch {b}: alloc {i}: gpu {go[i]:#x} oracle {out[i]:#x}"
            j = first_diff(from_dev(dst), st)
            assert j is None, f"batch {b}: free {j} status differs"
            if lock is not None:
                lock.batch(f, s)
                if b % state_every == 0:
                    assert np.array_equal(a.export_state(), lock.export_state()), f"batch {b}: state differs"
                    got, ref = a.stats(), lock.space()
                    assert (got["extent_bytes"], got["largest_free"]) == (ref["extent"], ref["largest_free"]), b
        gs = a.export_state()
        assert np.array_equal(gs, o.export_state()), "final state differs"
        if policy == "segfit":
            check_invariants(gs)
        ref = o.stats()
        got = a.stats()
        for k in ("alloc_ok", "alloc_fail", "free_ok", "free_fail", "used_bytes", "used_blocks",
                  "blocks", "requested_bytes", "bitmask"):
            assert got[k] == ref[k], (k, got[k], ref[k])
        sp = o.space()
        assert got["extent_bytes"] == sp["extent"] and got["largest_free"] == sp["largest_free"]
    if canary:
        torch.cuda.synchronize()
        assert canary_intact(guard), "the managed arena was written"
    return trace


def test_worked_examples(gpu_lib):
    """W1-W3 (hand-derived from Algorithms 4/5, tests/golden/worked_examples.txt)."""
    import torch

    from paper_2405_07079_gb300 import Allocator
    from test_oracle_pins import load_golden

    dev = torch.device("cuda")
    for case in load_golden():
        with Allocator(case["arena"], case["min_block"]) as a:
            for frees, sizes, expect in case["batches"]:
                f = to_dev(np.array(frees, np.uint64), dev)
                s = to_dev(np.array(sizes, np.uint64), dev)
                got = from_dev(a.step(f, s)) if sizes else np.zeros(0, np.uint64)
                if not sizes:
                    a.step(f, None)
                assert [int(x) for x in got] == expect, case["name"]
            if case.get("final") is not None:
                assert [int(x) for x in a.export_state()] == case["final"], case["name"]


@pytest.mark.parametrize("threads,ctas", [(32, 0), (128, 0), (256, 0), (512, 0), (1024, 0), (256, 1), (1024, 1),
                                          (1024, 2), (512, 8)])
def test_tiny_full(gpu_lib, threads, ctas):
    """1 MiB arena, 10,000 ops in batches of 64, canary arena untouched;
    every CTA width, with and without the gathering cluster."""
    from paper_2405_07079_gb300 import workloads as W

    _run(W.tiny(), threads=threads, state_every=16, canary=True, ctas=ctas)


@pytest.mark.parametrize("threads", [128, 1024])
@pytest.mark.parametrize("granules,batch,p_free", [(4096, 3000, 0.2), (8192, 64, 0.4), (8193, 64, 0.4)])
def test_small_record_tables(gpu_lib, threads, granules, batch, p_free):
    """Small arenas (1-2 MiB, record tables of 64-128 KiB, which the engine
    prefetches into L2 whole) with small batches (one launch, the engine
    gathering its frees) and batches large enough for the prep grid (at
    least 2,048 allocations, most of them failing in a full arena)."""
    from paper_2405_07079_gb300 import workloads as W

    wl = W.Workload("small-table", granules * 256, 256,
                    lambda: W.TinyRandom(n_ops=40 * batch if batch > 64 else 6000, batch=batch, p_free=p_free,
                                         hi=16 * KiB if batch > 64 else 64 * KiB))
    _run(wl, threads=threads, state_every=4, canary=True)


@pytest.mark.parametrize("batch", [1, 16])
def test_usage_workload(gpu_lib, batch):
    """The malloc-large stand-in (one op per batch, and batches of up to 16
    ops in sequential order): every result, the state, and the space report
    (extent, largest free block) against the oracle."""
    from paper_2405_07079_gb300 import workloads as W

    _run(W.usage(n_ops=2000, batch=batch), state_every=50 if batch == 1 else 10, canary=False)


@pytest.mark.parametrize("threads,ctas", [(128, 0), (1024, 0), (1024, 1), (256, 3)])
def test_large_reduced(gpu_lib, threads, ctas):
    from paper_2405_07079_gb300 import workloads as W

    wl = W.Workload("large-1GiB", 1 * GiB, 512, lambda: W.Lifetimes(n_ops=400_000, batch=8192, mean_life=300))
    _run(wl, threads=threads, state_every=5, ctas=ctas)


@pytest.mark.parametrize("ctas,na,per_batch", [(0, 4, 1), (0, 4096, 2), (4, 4, 1), (4, 4096, 1)])
def test_launches_per_batch(gpu_lib, ctas, na, per_batch):
    """Launches per batch with frees (counted by the handle): a small batch is
    gathered by the engine itself; a batch with many allocations gets the prep
    grid (gather + pre-filled failures) before the engine; a cluster does
    both in one launch.  Results equal the oracle's either way."""
    import numpy as np
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator

    dev = torch.device("cuda")
    ref = oracle.Oracle(1 << 24, 256)
    with Allocator(1 << 24, 256, threads=1024, ctas=ctas) as a:
        s1 = np.full(8, 4096, np.uint64)
        out = a.step(None, torch.from_numpy(s1.view(np.int64)).to(dev))
        ro, _ = ref.batch(np.zeros(0, np.uint64), s1)
        assert np.array_equal(out.cpu().numpy().view(np.uint64), ro)
        n0 = a.launches()
        s2 = np.full(na, 512, np.uint64)
        o2 = a.step(out[:4], torch.from_numpy(s2.view(np.int64)).to(dev))
        assert a.launches() - n0 == per_batch
        r2, _ = ref.batch(ro[:4], s2)
        assert np.array_equal(o2.cpu().numpy().view(np.uint64), r2)


def test_large_full(gpu_lib):
    """16 GiB arena, 10M ops in batches of 65,536: every result of every batch
    (the launch configuration the benchmark times); a real 16 GiB arena
    filled with the canary byte stays untouched."""
    from paper_2405_07079_gb300 import workloads as W

    _run(W.large(), threads=1024, state_every=50, canary=True)


def test_frag_reduced(gpu_lib):
    from paper_2405_07079_gb300 import workloads as W

    trace = _run(W.frag(n_fill=60_000, n_big=4000, batch=4096, arena=256 * MiB), threads=512, state_every=4)
    assert trace[-1][0].size > 0


def test_frag_full_returns_to_one_block(gpu_lib):
    """4 GiB, 1M x 4 KiB fill, free evens, 50k big, free all -> one block;
    a real 4 GiB arena filled with the canary byte stays untouched."""
    from paper_2405_07079_gb300 import workloads as W

    trace = _run(W.frag(), threads=1024, canary=True)
    fill = np.concatenate([t[2] for t in trace[:62]])
    assert np.array_equal(fill, np.arange(1_000_000, dtype=np.uint64) * 4096)


def test_frag_pow2_fill_all_big_fail(gpu_lib):
    """Fill with 2^20 x 4 KiB: the arena is exactly full with 4 KiB holes
    after the even frees, so every later request (class >= 13) fails."""
    from paper_2405_07079_gb300 import workloads as W

    trace = _run(W.frag(n_fill=1 << 20), threads=1024)
    big = [t for t in trace if t[1].size and t[1][0] != 4096]
    assert big and all((t[2] == FAIL).all() for t in big)


def test_edge_cases(gpu_lib):
    """Empty batches, size 0, oversize, whole-arena, invalid/duplicate frees."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator

    dev = torch.device("cuda")
    A, mb = 1 << 20, 256
    o = oracle.Oracle(A, mb)
    batches = [
        ([], []),
        ([], [0, A + 1, 1 << 63, FAIL, A]),          # only the whole-arena request succeeds
        ([0, 0, 1, 256, A, FAIL], [1]),               # duplicate, misaligned, interior, out of range
        ([0], []),                                    # double free across batches
        ([], [255, 256, 257, 4096, 65536, 1000]),
        ([256, 0, 512, 512, 1024], [A]),              # ragged frees incl. a free block
        ([], [1] * 5000),                             # many tiny requests
    ]
    with Allocator(A, mb, threads=256) as a:
        for f, s in batches:
            f = np.array(f, np.uint64)
            s = np.array(s, np.uint64)
            ro, rs = o.batch(f, s)
            dst = torch.empty(f.size, dtype=torch.uint8, device=dev)
            out = a.step(to_dev(f, dev) if f.size else None, to_dev(s, dev) if s.size else None, status=dst)
            if s.size:
                assert np.array_equal(from_dev(out), ro)
            assert np.array_equal(from_dev(dst), rs)
            assert np.array_equal(a.export_state(), o.export_state())


def test_free_slices_beyond_scratch(gpu_lib):
    """A batch with more frees than the scratch holds is applied in slices."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator

    dev = torch.device("cuda")
    A, mb = 64 * MiB, 256
    o = oracle.Oracle(A, mb)
    rng = np.random.default_rng(7)
    sizes = rng.integers(1, 8192, 3000).astype(np.uint64)
    with Allocator(A, mb, max_batch=100, threads=128) as a:
        ro, _ = o.batch(np.zeros(0, np.uint64), sizes)
        go = from_dev(a.step(None, to_dev(sizes, dev)))
        assert np.array_equal(go, ro)
        frees = ro[ro != FAIL][rng.permutation(int((ro != FAIL).sum()))]
        frees = np.concatenate([frees, frees[:50]])
        ro2, rs2 = o.batch(frees, sizes[:500])
        dst = torch.empty(frees.size, dtype=torch.uint8, device=dev)
        go2 = from_dev(a.step(to_dev(frees, dev), to_dev(sizes[:500], dev), status=dst))
        assert np.array_equal(go2, ro2) and np.array_equal(from_dev(dst), rs2)
        assert np.array_equal(a.export_state(), o.export_state())


def test_host_entry_point(gpu_lib):
    """hba_step_host (host buffers, copies inside) equals the device path."""
    import ctypes

    from paper_2405_07079_gb300 import Allocator, hba_step_host
    from paper_2405_07079_gb300 import workloads as W

    wl = W.tiny(n_ops=2000)
    trace, _ = oracle_trace(wl)
    with Allocator(wl.arena, wl.min_block) as a:
        for f, s, out, st in trace:
            f = np.ascontiguousarray(f)
            s = np.ascontiguousarray(s)
            go = np.empty(s.size, np.uint64)
            gst = np.empty(f.size, np.uint8)
            hba_step_host(a.h, f.ctypes.data if f.size else 0, f.size, gst.ctypes.data if f.size else 0,
                          s.ctypes.data if s.size else 0, s.size, go.ctypes.data if s.size else 0, 0)
            assert np.array_equal(go, out) and np.array_equal(gst, st)


def _pinned(a: np.ndarray):
    """A page-locked copy of a uint64 or uint8 array (a CPU torch tensor, kept
    alive by the caller) and its numpy view."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a).view(np.int64 if a.dtype == np.uint64 else np.uint8)).pin_memory()
    v = t.numpy()
    return t, (v.view(np.uint64) if a.dtype == np.uint64 else v)


@pytest.mark.parametrize("wl_name,max_batches", [("tiny", None), ("large", 8)])
def test_host_async_pipeline(gpu_lib, wl_name, max_batches):
    """hba_step_host_async with every batch of the trace in flight at once and
    one wait on the caller's stream at the end: every offset and status
    equals the oracle's.  A device-buffer hba_step on the caller's stream in
    the middle of the pipeline is ordered with the calls around it."""
    import torch

    from paper_2405_07079_gb300 import Allocator, hba_step_host_async
    from paper_2405_07079_gb300 import workloads as W

    wl = {"tiny": lambda: W.tiny(n_ops=3000), "large": W.large}[wl_name]()
    trace, o = oracle_trace(wl, max_batches)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    mid = len(trace) // 2
    keep, results = [], []
    with Allocator(wl.arena, wl.min_block) as a:
        for b, (f, s, out, st) in enumerate(trace):
            if b == mid:
                dst = torch.empty(f.size, dtype=torch.uint8, device=dev)
                go = a.step(to_dev(f, dev), to_dev(s, dev), status=dst) if s.size else None
                if not s.size:
                    a.step(to_dev(f, dev), None, status=dst)
                results.append(("dev", go, dst))
                continue
            tf, hf = _pinned(f)
            ts, hs = _pinned(s)
            to, ho = _pinned(np.zeros(s.size, np.uint64))
            tst, hst = _pinned(np.zeros(f.size, np.uint8))
            keep += [tf, ts, to, tst]
            hba_step_host_async(a.h, hf.ctypes.data if f.size else 0, f.size, hst.ctypes.data if f.size else 0,
                                hs.ctypes.data if s.size else 0, s.size, ho.ctypes.data if s.size else 0,
                                int(stream.cuda_stream))
            results.append(("host", ho, hst))
        stream.synchronize()
        for b, ((f, s, out, st), (kind, go, gst)) in enumerate(zip(trace, results)):
            if kind == "dev":
                go = from_dev(go) if go is not None else np.zeros(0, np.uint64)
                gst = from_dev(gst)
            i = first_diff(go, out)
            assert i is None, f"batch {b} ({kind}): alloc {i}: gpu {go[i]:#x} oracle {out[i]:#x}"
            assert first_diff(gst, st) is None, f"batch {b} ({kind}): free status differs"
        assert np.array_equal(a.export_state(), o.export_state())


def test_host_async_in_a_cuda_graph(gpu_lib):
    """While the stream is captured, hba_step_host_async records its copies
    and the batch on it; replaying the graph applies the batch like a direct
    call, and the pipelined form carries on from that state."""
    import torch

    from paper_2405_07079_gb300 import Allocator, hba_step_host_async
    from paper_2405_07079_gb300 import workloads as W

    wl = W.tiny(n_ops=400)
    trace, _ = oracle_trace(wl, 3)
    (f0, s0, out0, _), (f1, s1, out1, st1) = trace[0], trace[1]
    assert f0.size == 0 and s0.size and s1.size
    with Allocator(wl.arena, wl.min_block) as a:
        ts, hs = _pinned(s0)
        to, ho = _pinned(np.zeros(s0.size, np.uint64))
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
            hba_step_host_async(a.h, 0, 0, 0, hs.ctypes.data, s0.size, ho.ctypes.data, int(cap.cuda_stream))
        torch.cuda.synchronize()
        assert a.stats()["alloc_ok"] + a.stats()["alloc_fail"] == 0  # capturing ran nothing
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(ho, out0)
        tf1, hf1 = _pinned(f1)
        ts1, hs1 = _pinned(s1)
        to1, ho1 = _pinned(np.zeros(s1.size, np.uint64))
        tst1, hst1 = _pinned(np.zeros(f1.size, np.uint8))
        stream = torch.cuda.current_stream()
        hba_step_host_async(a.h, hf1.ctypes.data if f1.size else 0, f1.size, hst1.ctypes.data if f1.size else 0,
                            hs1.ctypes.data, s1.size, ho1.ctypes.data, int(stream.cuda_stream))
        stream.synchronize()
        assert np.array_equal(ho1, out1) and np.array_equal(hst1, st1)


def test_multi_arena_matches_per_arena_oracle(gpu_lib):
    """Independent arenas in one launch: arena i's results equal a single-arena
    oracle run of arena i's sub-trace."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import MultiAllocator
    from paper_2405_07079_gb300 import workloads as W

    dev = torch.device("cuda")
    rng = np.random.default_rng(11)
    n = 37
    sizes_a = (rng.integers(1, 64, n) * 256 * 1024 + rng.integers(0, 4, n) * 256).astype(np.uint64)
    mb = 256
    orcs = [oracle.Oracle(int(x), mb) for x in sizes_a]
    clients = [W.Lifetimes(n_ops=10**9, batch=int(rng.integers(0, 700)), mean_life=200,
                           seed=W.BASE_SEED + 100 + i, scale=float(x) / (16 * GiB), min_size=256)
               for i, x in enumerate(sizes_a)]
    for threads in (32, 64, 256):
        m = MultiAllocator(sizes_a, mb, max_total_frees=1 << 16)
        m.set_shape(threads)
        orcs = [oracle.Oracle(int(x), mb) for x in sizes_a]
        clients = [W.Lifetimes(n_ops=10**9, batch=int(rng.integers(0, 700)), mean_life=200,
                               seed=W.BASE_SEED + 100 + i, scale=float(x) / (16 * GiB), min_size=256)
                   for i, x in enumerate(sizes_a)]
        for b in range(12):
            fr, sz, exp_o, exp_s = [], [], [], []
            for i in range(n):
                f, s = clients[i].next_batch()
                ro, rs = orcs[i].batch(f, s)
                clients[i].feed(ro)
                fr.append(f); sz.append(s); exp_o.append(ro); exp_s.append(rs)
            frow = np.concatenate([[0], np.cumsum([x.size for x in fr])]).astype(np.uint32)
            arow = np.concatenate([[0], np.cumsum([x.size for x in sz])]).astype(np.uint32)
            F = np.concatenate(fr).astype(np.uint64)
            S = np.concatenate(sz).astype(np.uint64)
            out = torch.empty(S.size, dtype=torch.int64, device=dev)
            st = torch.empty(F.size, dtype=torch.uint8, device=dev)
            m.step(to_dev(frow.view(np.int32), dev), to_dev(F, dev), to_dev(arow.view(np.int32), dev),
                   to_dev(S, dev), out, st)
            assert np.array_equal(from_dev(out), np.concatenate(exp_o)), f"threads {threads} batch {b}"
            assert np.array_equal(from_dev(st), np.concatenate(exp_s))
        for i in range(n):
            assert np.array_equal(m.export_state(i), orcs[i].export_state()), i
        m.close()


@pytest.mark.parametrize("threads", [32, 128])
def test_batched_generator_matches_per_arena_oracles(gpu_lib, threads):
    """The batched workload (uneven arenas, U{0..2048} requests per arena per
    batch) in one multi-arena launch per batch equals, arena by arena, the
    oracle applied to that arena's sub-trace."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import MultiAllocator
    from paper_2405_07079_gb300 import workloads as W

    dev = torch.device("cuda")
    A = W.multi_arena_sizes(48, lo=1 << 20, hi=16 << 20)
    gen = W.MultiLifetimes(A, n_batches=12, mean_life=300)
    orcs = [oracle.Oracle(int(a), 256) for a in A]
    ma = MultiAllocator(A, 256, max_total_frees=48 * 2048 + 1)
    ma.set_shape(threads, 0, 0)
    try:
        for b in range(12):
            frow, f, arow, s = gen.next_batch()
            exp_o, exp_s = [], []
            for i in range(A.size):
                o, st = orcs[i].batch(f[frow[i]:frow[i + 1]], s[arow[i]:arow[i + 1]])
                exp_o.append(o)
                exp_s.append(st)
            out = torch.empty(s.size, dtype=torch.int64, device=dev)
            st = torch.empty(f.size, dtype=torch.uint8, device=dev)
            ma.step(to_dev(frow.view(np.int32), dev), to_dev(f, dev), to_dev(arow.view(np.int32), dev),
                    to_dev(s, dev), out, st)
            got = from_dev(out)
            assert np.array_equal(got, np.concatenate(exp_o)), f"batch {b}"
            assert np.array_equal(from_dev(st), np.concatenate(exp_s)), f"batch {b}"
            gen.feed(got)
        for i in range(A.size):
            assert np.array_equal(ma.export_state(i), orcs[i].export_state()), i
    finally:
        ma.close()


def _multi_oracle_trace(A, n_batches, max_ops, mean_life, mb=256, policy="segfit"):
    """The batched workload over arenas A, closed loop against one oracle
    per arena: [(frow, frees, arow, sizes, out, status)], and the oracles."""
    import oracle
    from paper_2405_07079_gb300 import workloads as W

    gen = W.MultiLifetimes(A, n_batches=n_batches, max_ops=max_ops, mean_life=mean_life)
    orcs = [oracle.Oracle(int(a), mb, policy) for a in A]
    trace = []
    while (b := gen.next_batch()) is not None:
        frow, f, arow, s = b
        outs, sts = [], []
        for i in range(A.size):
            o, st = orcs[i].batch(f[frow[i]:frow[i + 1]], s[arow[i]:arow[i + 1]])
            outs.append(o)
            sts.append(st)
        out, st = np.concatenate(outs), np.concatenate(sts)
        gen.feed(out)
        trace.append((frow, f, arow, s, out, st))
    return trace, orcs


def _multi_replay(A, trace, orcs, threads, ctas, mb=256, canaries=0, policy="segfit"):
    """Replay a batched trace through one multi-arena handle of the given
    launch shape: every offset and free status of every batch, and every
    arena's final state, equal the per-arena oracles'.  The first
    ``canaries`` arenas get a real buffer of their size filled with the
    canary byte, which must stay untouched."""
    import torch

    from _helpers import canary_intact
    from paper_2405_07079_gb300 import MultiAllocator

    dev = torch.device("cuda")
    guards = [torch.full((int(A[i]),), 0xA5, dtype=torch.uint8, device=dev) for i in range(canaries)]
    m = MultiAllocator(A, mb, max_total_frees=max(1, max(t[1].size for t in trace)), policy=policy)
    m.set_shape(threads, ctas, 0)
    try:
        for b, (frow, f, arow, s, out, st) in enumerate(trace):
            dout = torch.empty(max(1, s.size), dtype=torch.int64, device=dev)
            dst = torch.empty(max(1, f.size), dtype=torch.uint8, device=dev)
            m.step(to_dev(frow.view(np.int32), dev), to_dev(f, dev), to_dev(arow.view(np.int32), dev),
                   to_dev(s, dev), dout, dst)
            i = first_diff(from_dev(dout)[:s.size], out)
            assert i is None, f"shape {threads},{ctas} batch {b}: alloc {i}"
            assert first_diff(from_dev(dst)[:f.size], st) is None, f"shape {threads},{ctas} batch {b}: frees"
        for i in range(A.size):
            assert np.array_equal(m.export_state(i), orcs[i].export_state()), (threads, ctas, i)
        torch.cuda.synchronize()
        assert all(canary_intact(g) for g in guards), "a managed arena was written"
    finally:
        m.close()


@pytest.mark.parametrize("threads,ctas", [(32, 0), (32, 200), (128, 608), (256, 0)])
def test_multi_arena_large_grids(gpu_lib, threads, ctas):
    """2,700 arenas of 1-4 MiB, so that the launch shapes the full batched
    configuration uses all run: warp mode with more CTAs than two per SM
    (k_multi_warp built for four CTAs per SM), warp mode with 200 CTAs
    looping over the arenas, 608 CTAs of 128 threads looping over the
    arenas, and one CTA of 256 threads per arena."""
    from paper_2405_07079_gb300 import workloads as W

    A = W.multi_arena_sizes(2700, lo=1 << 20, hi=4 << 20)
    trace, orcs = _multi_oracle_trace(A, n_batches=8, max_ops=512, mean_life=300)
    _multi_replay(A, trace, orcs, threads, ctas, canaries=4)


@pytest.mark.parametrize("threads,ctas", [(32, 0), (128, 608)])
def test_tlsf_multi_arena_large_grids(gpu_lib, threads, ctas):
    """TLSF over 2,700 arenas of 1-4 MiB: warp mode with more CTAs than two
    per SM (four arenas per CTA, the build for four CTAs per SM), and 608
    CTAs of 128 threads looping over the arenas (the shape family the
    autotuner picks for TLSF on the full batched configuration)."""
    from paper_2405_07079_gb300 import workloads as W

    A = W.multi_arena_sizes(2700, lo=1 << 20, hi=4 << 20)
    trace, orcs = _multi_oracle_trace(A, n_batches=8, max_ops=512, mean_life=300, policy="tlsf")
    _multi_replay(A, trace, orcs, threads, ctas, canaries=2, policy="tlsf")


def test_multi_arena_full_config_autotuned_shape(gpu_lib):
    """The full batched configuration's arenas (4,096, log-uniform 64 MiB -
    1 GiB) and request counts (U{0..2048} per arena per batch), three batches,
    at the shape the autotuner picks on GB300 (warp mode, 608 CTAs): every
    arena against its own oracle; two arenas get canary buffers."""
    from paper_2405_07079_gb300 import workloads as W

    A = W.multi_arena_sizes()
    trace, orcs = _multi_oracle_trace(A, n_batches=3, max_ops=2048, mean_life=1000)
    assert sum(t[3].size for t in trace) > 7_000_000
    _multi_replay(A, trace, orcs, 32, 608, canaries=2)


def test_multi_step_host_async_matches_oracles(gpu_lib):
    """hba_multi_step_host_async: the batched form from pinned host buffers,
    three calls in flight before the host reads the first results (the two
    staging slots are reused while earlier calls' copies are still queued):
    every offset and free status equals the per-arena oracles', and a handle
    made without staging refuses the call."""
    import torch

    from paper_2405_07079_gb300 import HbaError, MultiAllocator, hba_multi_step_host_async
    from paper_2405_07079_gb300 import workloads as W

    A = W.multi_arena_sizes(300, lo=1 << 20, hi=8 << 20)
    trace, orcs = _multi_oracle_trace(A, n_batches=9, max_ops=1024, mean_life=200)
    nf_max = max(t[1].size for t in trace)
    na_max = max(t[3].size for t in trace)
    m = MultiAllocator(A, 256, max_total_frees=nf_max, max_total_allocs=na_max)
    stream = torch.cuda.current_stream()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    try:
        keep = []
        for frow, f, arow, s, out, st in trace:
            hfr, har = pin(frow.view(np.int32)), pin(arow.view(np.int32))
            hf, hs = pin(f.view(np.int64)), pin(s.view(np.int64))
            ho = torch.empty(max(1, s.size), dtype=torch.int64).pin_memory()
            hst = torch.empty(max(1, f.size), dtype=torch.uint8).pin_memory()
            hba_multi_step_host_async(m.h, hfr.data_ptr(), hf.data_ptr() if f.size else 0, f.size, har.data_ptr(),
                                      hs.data_ptr() if s.size else 0, s.size, ho.data_ptr() if s.size else 0,
                                      hst.data_ptr() if f.size else 0, int(stream.cuda_stream))
            keep.append((hfr, har, hf, hs, ho, hst, out, st))
        stream.synchronize()
        for b, (_, _, _, _, ho, hst, out, st) in enumerate(keep):
            assert np.array_equal(ho.numpy().view(np.uint64)[:out.size], out), f"batch {b}"
            assert np.array_equal(hst.numpy()[:st.size], st), f"batch {b} frees"
        for i in range(A.size):
            assert np.array_equal(m.export_state(i), orcs[i].export_state()), i
    finally:
        m.close()
    plain = MultiAllocator(A[:4], 256, max_total_frees=16)
    z = torch.zeros(8, dtype=torch.int32).pin_memory()
    with pytest.raises(HbaError):
        hba_multi_step_host_async(plain.h, z.data_ptr(), 0, 0, z.data_ptr(), 0, 0, 0, 0, 0)
    plain.close()


def test_multi_step_host_async_in_a_captured_graph(gpu_lib):
    """hba_multi_step_host_async captured into a CUDA graph: capturing runs
    nothing; each replay applies the captured batch from the same pinned
    host buffers (rewritten between replays) and writes the results back;
    results equal the per-arena oracles batch after batch."""
    import torch

    from paper_2405_07079_gb300 import MultiAllocator, hba_multi_step_host_async
    from paper_2405_07079_gb300 import workloads as W

    A = W.multi_arena_sizes(64, lo=1 << 20, hi=4 << 20)
    trace, orcs = _multi_oracle_trace(A, n_batches=4, max_ops=64, mean_life=50)
    nf_max = max(t[1].size for t in trace)
    na_max = max(t[3].size for t in trace)
    m = MultiAllocator(A, 256, max_total_frees=max(1, nf_max), max_total_allocs=na_max)
    try:
        hfr = torch.zeros(A.size + 1, dtype=torch.int32).pin_memory()
        har = torch.zeros(A.size + 1, dtype=torch.int32).pin_memory()
        hf = torch.zeros(max(1, nf_max), dtype=torch.int64).pin_memory()
        hs = torch.zeros(max(1, na_max), dtype=torch.int64).pin_memory()
        ho = torch.zeros(max(1, na_max), dtype=torch.int64).pin_memory()
        hst = torch.zeros(max(1, nf_max), dtype=torch.uint8).pin_memory()
        # a graph replays fixed sizes: capture one call per distinct (nf, na) of the trace
        graphs = {}
        cap = torch.cuda.Stream()
        for frow, f, arow, s, out, st in trace:
            key = (f.size, s.size)
            if key in graphs:
                continue
            g = torch.cuda.CUDAGraph()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
                hba_multi_step_host_async(m.h, hfr.data_ptr(), hf.data_ptr(), f.size, har.data_ptr(),
                                          hs.data_ptr(), s.size, ho.data_ptr(), hst.data_ptr(),
                                          int(cap.cuda_stream))
            graphs[key] = g
        torch.cuda.synchronize()
        assert m.stats()["alloc_ok"] + m.stats()["alloc_fail"] == 0  # capturing ran nothing
        for b, (frow, f, arow, s, out, st) in enumerate(trace):
            hfr.numpy()[:] = frow.view(np.int32)
            har.numpy()[:] = arow.view(np.int32)
            hf.numpy()[:f.size] = f.view(np.int64)
            hs.numpy()[:s.size] = s.view(np.int64)
            graphs[(f.size, s.size)].replay()
            torch.cuda.synchronize()
            assert np.array_equal(ho.numpy().view(np.uint64)[:s.size], out), f"batch {b}"
            assert np.array_equal(hst.numpy()[:f.size], st), f"batch {b} frees"
        for i in range(A.size):
            assert np.array_equal(m.export_state(i), orcs[i].export_state()), i
    finally:
        m.close()


def test_calls_on_two_streams_are_ordered(gpu_lib):
    """Batches issued back to back on two different streams, with no host
    synchronisation between them: the handle orders the second after the
    first (its internal event), so results equal the oracle's."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator, workloads as W

    dev = torch.device("cuda")
    wl = W.Workload("life", 1 << 28, 512, lambda: W.Lifetimes(n_ops=60_000, batch=2048, mean_life=40))
    trace, _ = oracle_trace(wl)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    with Allocator(wl.arena, wl.min_block) as a:
        for b, (f, s, out, st) in enumerate(trace):
            stream = streams[b % 2]
            with torch.cuda.stream(stream):
                df, ds = to_dev(f, dev), to_dev(s, dev)
                dst = torch.empty(f.size, dtype=torch.uint8, device=dev)
                o = torch.empty(max(s.size, 1), dtype=torch.int64, device=dev)
                a.step(df if f.size else None, ds if s.size else None, out=o, status=dst, stream=stream)
                outs.append((o, dst, df, ds))
        torch.cuda.synchronize()
        for b, ((o, dst, _, _), (f, s, out, st)) in enumerate(zip(outs, trace)):
            assert np.array_equal(from_dev(o)[:s.size], out), f"batch {b}"
            assert np.array_equal(from_dev(dst), st), f"batch {b} frees"
        ref = oracle.Oracle(wl.arena, wl.min_block)
        for f, s, _, _ in trace:
            ref.batch(f, s)
        assert np.array_equal(a.export_state(), ref.export_state())


# ---- two-level segregated fit (§5.2) -----------------------------------------


def test_tlsf_worked_examples(gpu_lib):
    """The hand-derived TLSF examples through the GPU kernel."""
    import sys

    import torch

    from paper_2405_07079_gb300 import Allocator

    sys.path.insert(0, __import__("os").path.dirname(__file__))
    from test_oracle_pins import load_tlsf_golden

    dev = torch.device("cuda")
    for case in load_tlsf_golden():
        with Allocator(case["arena"], case["min_block"], policy="tlsf") as a:
            for frees, sizes, expect in case["batches"]:
                f = np.array(frees, np.uint64)
                st = torch.empty(f.size, dtype=torch.uint8, device=dev)
                out = a.step(to_dev(f, dev) if f.size else None, to_dev(np.array(sizes, np.uint64), dev), status=st)
                assert [int(x) for x in from_dev(out)] == expect, case["name"]
                assert not from_dev(st).any()
            assert [int(x) for x in a.export_state()] == case["final"], case["name"]


def test_tlsf_tiny_full(gpu_lib):
    from paper_2405_07079_gb300 import workloads as W

    _run(W.tiny(), state_every=8, canary=True, policy="tlsf")


@pytest.mark.parametrize("batch", [1, 16])
def test_tlsf_usage_workload(gpu_lib, batch):
    from paper_2405_07079_gb300 import workloads as W

    _run(W.usage(n_ops=2000, batch=batch), state_every=50 if batch == 1 else 10, policy="tlsf")


def test_tlsf_large_reduced(gpu_lib):
    """Batches of 8,192 requests on a 1 GiB arena: allocation windows of 32
    with long runs of failures, frees with merges."""
    from paper_2405_07079_gb300 import workloads as W

    wl = W.Workload("large-1GiB", 1 * GiB, 512, lambda: W.Lifetimes(n_ops=200_000, batch=8192, mean_life=300))
    _run(wl, state_every=5, policy="tlsf")


def test_tlsf_large_full(gpu_lib):
    """Two-level segregated fit on the full large trace (16 GiB arena, 10M
    ops in batches of 65,536) through the batch engine, the launch
    configuration the benchmark times: every result of every batch, the
    state every 50 batches, and a 16 GiB canary arena left untouched."""
    from paper_2405_07079_gb300 import workloads as W

    _run(W.large(), threads=1024, state_every=50, canary=True, policy="tlsf")


def test_tlsf_frag_reduced(gpu_lib):
    from paper_2405_07079_gb300 import workloads as W

    _run(W.frag(n_fill=40_000, n_big=3000, batch=4096, arena=256 * MiB), state_every=4, policy="tlsf")


def test_tlsf_edge_cases(gpu_lib):
    """Size 0, sizes above the arena, misaligned, unknown, interior and
    duplicate frees, an empty batch, and a batch that empties the arena."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator

    dev = torch.device("cuda")
    A, mb = 1 << 20, 256
    o = oracle.Oracle(A, mb, "tlsf")
    u = lambda *v: np.array(v, dtype=np.uint64)
    batches = [
        (u(), u(0, 1, A, A + 1, 1 << 63, 300, 70000)),
        (u(), u()),
        (u(1, 256 + 8, 12345 * 256, 0, 0, 512), u(256)),
        (u(A, A + 256, 1 << 40), u(5000)),
    ]
    with Allocator(A, mb, policy="tlsf") as a:
        for f, s_ in batches:
            ro, rs = o.batch(f, s_)
            st = torch.empty(f.size, dtype=torch.uint8, device=dev)
            out = a.step(to_dev(f, dev) if f.size else None, to_dev(s_, dev) if s_.size else None, status=st)
            if s_.size:
                assert np.array_equal(from_dev(out), ro)
            assert np.array_equal(from_dev(st), rs)
        sizes_ = oracle.decode_state(o.export_state(), "tlsf")["blocks"]
        used = u(*[off for off, _, fr in sizes_ if not fr])
        ro, rs = o.batch(used, u(A))
        st = torch.empty(used.size, dtype=torch.uint8, device=dev)
        out = a.step(to_dev(used, dev), to_dev(u(A), dev), status=st)
        assert np.array_equal(from_dev(out), ro) and ro[0] == 0 and not rs.any()
        assert np.array_equal(a.export_state(), o.export_state())
        got, sp = a.stats(), o.space()
        assert got["extent_bytes"] == sp["extent"] == A and got["largest_free"] == sp["largest_free"] == 0


def test_tlsf_host_entry_points_and_serving_refusal(gpu_lib):
    """The host-buffer calls and the no-scratch entry point run TLSF handles;
    the serving loop (segregated fit only) rejects them."""
    import torch

    from paper_2405_07079_gb300 import Allocator, HbaError, hba_step_host, hba_step_static
    from paper_2405_07079_gb300 import workloads as W

    wl = W.tiny(n_ops=1500)
    trace, orc = oracle_trace(wl, policy="tlsf")
    dev = torch.device("cuda")
    with Allocator(wl.arena, wl.min_block, policy="tlsf") as a, \
            Allocator(wl.arena, wl.min_block, policy="tlsf", max_batch=1) as b:
        for f, s, out, st in trace:
            f = np.ascontiguousarray(f)
            s = np.ascontiguousarray(s)
            go = np.empty(s.size, np.uint64)
            gst = np.empty(f.size, np.uint8)
            hba_step_host(a.h, f.ctypes.data if f.size else 0, f.size, gst.ctypes.data if f.size else 0,
                          s.ctypes.data if s.size else 0, s.size, go.ctypes.data if s.size else 0, 0)
            assert np.array_equal(go, out) and np.array_equal(gst, st)
            dst = torch.empty(f.size, dtype=torch.uint8, device=dev)
            dout = torch.empty(s.size, dtype=torch.int64, device=dev)
            df, ds = to_dev(f, dev), to_dev(s, dev)  # kept alive until the call has run
            hba_step_static(b.h, df.data_ptr() if f.size else 0, f.size, dst.data_ptr() if f.size else 0,
                            ds.data_ptr() if s.size else 0, s.size, dout.data_ptr() if s.size else 0,
                            int(torch.cuda.current_stream().cuda_stream))
            torch.cuda.synchronize()
            if s.size:
                assert np.array_equal(from_dev(dout), out)
            if f.size:
                assert np.array_equal(from_dev(dst), st)
        assert np.array_equal(b.export_state(), orc.export_state())
        assert np.array_equal(a.export_state(), orc.export_state())
        from paper_2405_07079_gb300 import serve, workloads
        arr = workloads.serving_arrivals(1e5, 0.001)
        with pytest.raises(HbaError):
            serve(a, arr)


@pytest.mark.parametrize("shape", [(32, 0), (32, 40), (64, 152), (128, 0), (256, 0)])
def test_tlsf_multi_arena_matches_per_arena_oracles(gpu_lib, shape):
    """Independent TLSF arenas in one launch of the batch engine with the
    two-level lists, one warp each (32 threads, four arenas per CTA) or one
    CTA each; a grid smaller than it needs makes CTAs loop over arenas.
    Arena i's results equal a TLSF oracle run of arena i's sub-trace."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import MultiAllocator
    from paper_2405_07079_gb300 import workloads as W

    dev = torch.device("cuda")
    rng = np.random.default_rng(21)
    n = 203
    sizes_a = (rng.integers(1, 64, n) * 256 * 1024 + rng.integers(0, 4, n) * 256).astype(np.uint64)
    mb = 256
    m = MultiAllocator(sizes_a, mb, max_total_frees=1 << 18, policy="tlsf")
    m.set_shape(*shape)
    orcs = [oracle.Oracle(int(x), mb, "tlsf") for x in sizes_a]
    clients = [W.Lifetimes(n_ops=10**9, batch=int(rng.integers(0, 700)), mean_life=200,
                           seed=W.BASE_SEED + 300 + i, scale=float(x) / (16 * GiB), min_size=256)
               for i, x in enumerate(sizes_a)]
    for b in range(12):
        fr, sz, exp_o, exp_s = [], [], [], []
        for i in range(n):
            f, s_ = clients[i].next_batch()
            ro, rs = orcs[i].batch(f, s_)
            clients[i].feed(ro)
            fr.append(f); sz.append(s_); exp_o.append(ro); exp_s.append(rs)
        frow = np.concatenate([[0], np.cumsum([x.size for x in fr])]).astype(np.uint32)
        arow = np.concatenate([[0], np.cumsum([x.size for x in sz])]).astype(np.uint32)
        F = np.concatenate(fr).astype(np.uint64)
        S = np.concatenate(sz).astype(np.uint64)
        out = torch.empty(S.size, dtype=torch.int64, device=dev)
        st = torch.empty(F.size, dtype=torch.uint8, device=dev)
        m.step(to_dev(frow.view(np.int32), dev), to_dev(F, dev), to_dev(arow.view(np.int32), dev),
               to_dev(S, dev), out, st)
        assert np.array_equal(from_dev(out), np.concatenate(exp_o)), f"batch {b}"
        assert np.array_equal(from_dev(st), np.concatenate(exp_s))
    for i in range(n):
        assert np.array_equal(m.export_state(i), orcs[i].export_state()), i
    st_ = m.stats()
    assert st_["alloc_ok"] == sum(o.stats()["alloc_ok"] for o in orcs)
    assert st_["extent_bytes"] == sum(o.space()["extent"] for o in orcs)
    m.close()


# ---- sequential fits on address-sorted lists (§3.1, §4) ------------------------


def _hal_trace(wl, fit, max_batches=None):
    import oracle

    o = oracle.HalOracle(wl.arena, wl.min_block, fit)
    cl = wl.make()
    trace = []
    while max_batches is None or len(trace) < max_batches:
        b = cl.next_batch()
        if b is None:
            break
        out, st = o.batch(*b)
        cl.feed(out)
        trace.append((b[0], b[1], out, st))
    return trace, o


def _run_fit(trace, o, arena, min_block, fit, state_every=0):
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator

    dev = torch.device("cuda")
    lock = oracle.HalOracle(arena, min_block, fit) if state_every else None
    with Allocator(arena, min_block, policy=fit) as a:
        for b, (f, s, out, st) in enumerate(trace):
            dst = torch.empty(f.size, dtype=torch.uint8, device=dev)
            go = a.step(to_dev(f, dev) if f.size else None, to_dev(s, dev) if s.size else None, status=dst)
            if s.size:
                i = first_diff(from_dev(go), out)
                assert i is None, f"{fit} batch {b}: alloc {i}"
            assert first_diff(from_dev(dst), st) is None, f"{fit} batch {b}: free status"
            if lock is not None:
                lock.batch(f, s)
                if b % state_every == 0:
                    assert np.array_equal(a.export_state(), lock.export_state()), f"{fit} batch {b}: state"
        assert np.array_equal(a.export_state(), o.export_state()), f"{fit}: final state"
        got, ref = a.stats(), o.stats()
        for k in ("alloc_ok", "alloc_fail", "free_ok", "free_fail", "used_bytes", "used_blocks", "blocks",
                  "requested_bytes", "largest_free"):
            assert got[k] == ref[k], (fit, k, got[k], ref[k])
        assert got["extent_bytes"] == ref["extent"]


@pytest.mark.parametrize("fit", ["first", "next", "best"])
def test_fits_worked_examples(gpu_lib, fit):
    import sys

    import torch

    from paper_2405_07079_gb300 import Allocator

    sys.path.insert(0, __import__("os").path.dirname(__file__))
    from test_oracle_pins import load_hal_golden

    dev = torch.device("cuda")
    for case in [c for c in load_hal_golden() if c["fit"] == fit]:
        with Allocator(case["arena"], case["min_block"], policy=fit) as a:
            for frees, sizes, expect, expect_st in case["batches"]:
                f = np.array(frees, np.uint64)
                s_ = np.array(sizes, np.uint64)
                st = torch.empty(f.size, dtype=torch.uint8, device=dev)
                out = a.step(to_dev(f, dev) if f.size else None, to_dev(s_, dev) if s_.size else None, status=st)
                if s_.size:
                    assert [int(x) for x in from_dev(out)] == expect, case["name"]
                assert [int(x) for x in from_dev(st)] == expect_st, case["name"]
            assert [int(x) for x in a.export_state()] == case["final"], case["name"]


@pytest.mark.parametrize("fit", ["first", "next", "best"])
def test_fits_tiny_and_usage(gpu_lib, fit):
    from paper_2405_07079_gb300 import workloads as W

    for wl, every in ((W.tiny(n_ops=4000), 8), (W.usage(n_ops=1500, batch=16), 10)):
        trace, o = _hal_trace(wl, fit)
        _run_fit(trace, o, wl.arena, wl.min_block, fit, state_every=every)


@pytest.mark.parametrize("fit", ["first", "next", "best"])
def test_fits_lifetimes_large_lists(gpu_lib, fit):
    """Batches of 4,096 requests on a 256 MiB arena: free lists of hundreds
    to thousands of entries (multi-step scans and shifts), long failure runs."""
    from paper_2405_07079_gb300 import workloads as W

    wl = W.Workload("life", 256 * MiB, 512, lambda: W.Lifetimes(n_ops=60_000, batch=4096, mean_life=400))
    trace, o = _hal_trace(wl, fit)
    _run_fit(trace, o, wl.arena, wl.min_block, fit, state_every=3)


@pytest.mark.parametrize("fit", ["first", "next", "best"])
def test_fits_arrays_past_shared_memory(gpu_lib, fit):
    """The kernel keeps the free and used arrays in shared memory while each
    holds at most 4,096 entries: a batch whose allocations push the used
    array past that (the arrays move to global memory mid-batch), batches
    that start in global memory, and batches that start in shared memory
    again after frees; partial frees in between."""
    import oracle

    rng = np.random.default_rng({"first": 31, "next": 32, "best": 33}[fit])
    arena, mb = 16 * MiB, 256
    o = oracle.HalOracle(arena, mb, fit)
    held, trace = [], []

    def batch(frees, sizes):
        f = np.array(frees, np.uint64)
        s_ = np.array(sizes, np.uint64)
        out, st = o.batch(f, s_)
        trace.append((f, s_, out, st))
        return [int(x) for x in out if x != FAIL]

    small = lambda n: (rng.integers(1, 9, n) * mb - rng.integers(0, mb, n)).tolist()
    held += batch([], small(3000))
    held += batch([], small(2500))                        # 5,500 used entries: past 4,096 mid-batch
    rng.shuffle(held)
    fr, held = held[:2000], held[2000:]
    held += batch(fr, small(800))                         # starts in global memory
    rng.shuffle(held)
    fr, held = held[:3900], held[3900:]
    part = [h + mb for h in held[:150]]                    # partial frees: keep the first unit
    held += batch(fr + part, small(300))
    held += batch([], small(4500))                        # starts in shared memory, grows past it again
    rng.shuffle(held)
    batch(held, small(50))
    assert max(len(t[1]) for t in trace) >= 2500
    _run_fit(trace, o, arena, mb, fit, state_every=1)


@pytest.mark.parametrize("fit", ["first", "next", "best"])
def test_fits_partial_and_invalid_frees(gpu_lib, fit):
    """Random batches whose frees name block starts, interior granules
    (partial deallocation), misaligned and unknown offsets."""
    rng = np.random.default_rng({"first": 5, "next": 6, "best": 7}[fit])
    import oracle

    A, mb = 8 * MiB, 4096
    o = oracle.HalOracle(A, mb, fit)
    held, trace = [], []
    for _ in range(300):
        frees = []
        for _ in range(int(rng.integers(0, 24))):
            if held and rng.random() < 0.8:
                h = held[int(rng.integers(0, len(held)))]
                frees.append(h + mb * int(rng.integers(0, 4)) if rng.random() < 0.35 else h)
            else:
                frees.append(int(rng.integers(0, A // mb + 4)) * mb + int(rng.choice([0, 0, 8])))
        sizes = (rng.integers(1, 64, int(rng.integers(0, 40))) * 4096 - rng.integers(0, 4096, 1)).astype(np.uint64)
        f = np.array(frees, np.uint64)
        out, st = o.batch(f, sizes)
        trace.append((f, sizes, out, st))
        held = [h for h in held if h not in frees] + [int(x) for x in out if x != FAIL]
    o2 = oracle.HalOracle(A, mb, fit)
    for f, s, _, _ in trace:
        o2.batch(f, s)
    _run_fit(trace, o2, A, mb, fit, state_every=25)


def test_fits_multi_arena(gpu_lib):
    """Independent first/next/best-fit arenas, one CTA each, in one launch."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import MultiAllocator
    from paper_2405_07079_gb300 import workloads as W

    dev = torch.device("cuda")
    rng = np.random.default_rng(33)
    n = 41
    sizes_a = (rng.integers(1, 32, n) * 256 * 1024 + rng.integers(0, 4, n) * 256).astype(np.uint64)
    mb = 256
    for fit in ("first", "next", "best"):
        m = MultiAllocator(sizes_a, mb, max_total_frees=1 << 16, policy=fit)
        orcs = [oracle.HalOracle(int(x), mb, fit) for x in sizes_a]
        clients = [W.Lifetimes(n_ops=10**9, batch=int(rng.integers(0, 300)), mean_life=100,
                               seed=W.BASE_SEED + 500 + i, scale=float(x) / (16 * GiB), min_size=256)
                   for i, x in enumerate(sizes_a)]
        for b in range(8):
            fr, sz, exp_o, exp_s = [], [], [], []
            for i in range(n):
                f, s_ = clients[i].next_batch()
                ro, rs = orcs[i].batch(f, s_)
                clients[i].feed(ro)
                fr.append(f); sz.append(s_); exp_o.append(ro); exp_s.append(rs)
            frow = np.concatenate([[0], np.cumsum([x.size for x in fr])]).astype(np.uint32)
            arow = np.concatenate([[0], np.cumsum([x.size for x in sz])]).astype(np.uint32)
            F = np.concatenate(fr).astype(np.uint64)
            S = np.concatenate(sz).astype(np.uint64)
            out = torch.empty(S.size, dtype=torch.int64, device=dev)
            st = torch.empty(F.size, dtype=torch.uint8, device=dev)
            m.step(to_dev(frow.view(np.int32), dev), to_dev(F, dev), to_dev(arow.view(np.int32), dev),
                   to_dev(S, dev), out, st)
            assert np.array_equal(from_dev(out), np.concatenate(exp_o)), f"{fit} batch {b}"
            assert np.array_equal(from_dev(st), np.concatenate(exp_s))
        for i in range(n):
            assert np.array_equal(m.export_state(i), orcs[i].export_state()), (fit, i)
        m.close()


# ---- bitmask pool (§3.2) -------------------------------------------------------


def _run_bitmask(trace, o, pool, unit, state_every=0):
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator

    dev = torch.device("cuda")
    lock = oracle.BitmaskOracle(pool, unit) if state_every else None
    with Allocator(pool, unit, policy="bitmask") as a:
        for b, (f, s, out, st) in enumerate(trace):
            dst = torch.empty(f.size, dtype=torch.uint8, device=dev)
            go = a.step(to_dev(f, dev) if f.size else None, to_dev(s, dev) if s.size else None, status=dst)
            if s.size:
                i = first_diff(from_dev(go), out)
                assert i is None, f"batch {b}: alloc {i}"
            assert first_diff(from_dev(dst), st) is None, f"batch {b}: free status"
            if lock is not None:
                lock.batch(f, s)
                if b % state_every == 0:
                    assert np.array_equal(a.export_state(), lock.export_state()), f"batch {b}: state"
        assert np.array_equal(a.export_state(), o.export_state()), "final state"
        got, ref = a.stats(), o.stats()
        for k in ("alloc_ok", "alloc_fail", "free_ok", "free_fail", "used_bytes", "used_blocks", "blocks",
                  "requested_bytes", "largest_free"):
            assert got[k] == ref[k], (k, got[k], ref[k])
        assert got["extent_bytes"] == ref["extent"]


def test_bitmask_worked_examples(gpu_lib):
    import sys

    import torch

    from paper_2405_07079_gb300 import Allocator

    sys.path.insert(0, __import__("os").path.dirname(__file__))
    from test_oracle_pins import load_bitmask_golden

    dev = torch.device("cuda")
    for case in load_bitmask_golden():
        with Allocator(case["pool"], case["unit"], policy="bitmask") as a:
            for frees, sizes, expect, expect_st in case["batches"]:
                f = np.array(frees, np.uint64)
                s_ = np.array(sizes, np.uint64)
                st = torch.empty(f.size, dtype=torch.uint8, device=dev)
                out = a.step(to_dev(f, dev) if f.size else None, to_dev(s_, dev) if s_.size else None, status=st)
                if s_.size:
                    assert [int(x) for x in from_dev(out)] == expect, case["name"]
                assert [int(x) for x in from_dev(st)] == expect_st, case["name"]
            assert [int(x) for x in a.export_state()] == case["final"], case["name"]


@pytest.mark.parametrize("pool,unit,batch,hi", [(1 << 20, 8, 256, 520), (1000 * 8, 8, 16, 520),
                                                (786_432 * 16, 16, 2048, 1040), (1 << 20, 8, 256, 4096),
                                                (786_432 * 8, 8, 512, 32768)])
def test_bitmask_objects(gpu_lib, pool, unit, batch, hi):
    """Pools of 131,072 units, of 1,000 units (a partial last word), and of
    the largest size a pool may have (786,432 units): every result, the state
    and the counters against the oracle.  Objects reach 65 units, and in the
    last two cases 512 and 4,096 units (runs longer than one 128-bit window,
    §3.2's 1 kB = 128-bit example and beyond)."""
    import oracle
    from paper_2405_07079_gb300 import workloads as W

    wl = W.Workload("objects", pool, unit, lambda: W.TinyRandom(n_ops=30 * batch if batch > 16 else 3000, batch=batch,
                                                                p_free=0.45, lo=1, hi=hi))
    o = oracle.BitmaskOracle(pool, unit)
    cl = wl.make()
    trace = []
    while (b := cl.next_batch()) is not None:
        out, st = o.batch(*b)
        cl.feed(out)
        trace.append((b[0], b[1], out, st))
    o2 = oracle.BitmaskOracle(pool, unit)
    for f, s, _, _ in trace:
        o2.batch(f, s)
    _run_bitmask(trace, o2, pool, unit, state_every=max(1, len(trace) // 8))


@pytest.mark.parametrize("units,seed", [(4096, 0), (1000, 1), (8192, 2), (64 * 3, 3), (12288 * 64, 4)])
def test_bitmask_long_runs_fragmented(gpu_lib, units, seed):
    """Runs longer than 64 units in a pool fragmented around word
    boundaries: fill with small objects, free a random half (holes of every
    length, starting and ending anywhere in a word), then ask for runs of
    65 units up to the whole pool, interleaved with small objects and frees;
    finally free everything and take the whole pool in one request."""
    import oracle

    rng = np.random.default_rng(500 + seed)
    unit = 8
    pool = units * unit
    o = oracle.BitmaskOracle(pool, unit)
    held, trace = [], []

    def batch(frees, sizes):
        f = np.array(frees, np.uint64)
        s = np.array(sizes, np.uint64)
        out, st = o.batch(f, s)
        trace.append((f, s, out, st))
        return [int(x) for x in out if x != FAIL]

    for _ in range(6):  # fill with objects of 1-40 units
        held += batch([], rng.integers(1, 40 * unit, int(rng.integers(100, 400))).tolist())
    rng.shuffle(held)
    half = len(held) // 2
    batch(held[:half], [])
    held = held[half:]
    for _ in range(25):
        nf = int(rng.integers(0, min(len(held), 12) + 1))
        idx = rng.choice(len(held), nf, replace=False) if nf else []
        frees = [held[i] for i in idx]
        held = [h for i, h in enumerate(held) if i not in set(idx)]
        kinds = rng.random(int(rng.integers(1, 40)))
        sizes = [int(rng.integers(1, 65 * unit)) if r < 0.3 else
                 int(rng.integers(65 * unit, 700 * unit)) if r < 0.9 else
                 int(rng.integers(1, pool + unit)) for r in kinds]
        held += batch(frees, sizes)
    batch(held, [pool, unit, pool // 2])
    o2 = oracle.BitmaskOracle(pool, unit)
    for f, s, _, _ in trace:
        o2.batch(f, s)
    _run_bitmask(trace, o2, pool, unit, state_every=3)


def test_bitmask_invalid_frees_and_pool_limit(gpu_lib):
    """Misaligned, interior, repeated and out-of-pool frees; a pool one unit
    above the limit is refused at create."""
    import oracle
    from paper_2405_07079_gb300 import Allocator, HbaError

    rng = np.random.default_rng(8)
    pool, unit = 4096 * 8, 8
    o = oracle.BitmaskOracle(pool, unit)
    held, trace = [], []
    for _ in range(120):
        frees = []
        for _ in range(int(rng.integers(0, 20))):
            if held and rng.random() < 0.7:
                h = held[int(rng.integers(0, len(held)))]
                frees.append(h + int(rng.choice([0, 0, 0, unit, 3])))
            else:
                frees.append(int(rng.integers(0, pool // unit + 8)) * unit)
        sizes = rng.integers(0, 70 * unit, int(rng.integers(0, 30))).astype(np.uint64)
        f = np.array(frees, np.uint64)
        out, st = o.batch(f, sizes)
        trace.append((f, sizes, out, st))
        held = [h for h in held if h not in frees] + [int(x) for x in out if x != FAIL]
    o2 = oracle.BitmaskOracle(pool, unit)
    for f, s, _, _ in trace:
        o2.batch(f, s)
    _run_bitmask(trace, o2, pool, unit, state_every=10)
    with pytest.raises(HbaError):
        Allocator((786_432 + 1) * 8, 8, policy="bitmask")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bitmask_many_frees_with_repeats(gpu_lib, seed):
    """Batches of up to 900 frees (several chunks of the kernel's parallel
    free phase): neighbouring blocks freed together, blocks of up to 300
    units (several words), the same block named twice in one chunk and in
    different chunks, interior, misaligned and out-of-pool offsets; every
    status, result and the state against the oracle."""
    import oracle

    rng = np.random.default_rng(900 + seed)
    unit, units = 8, 64 * 700
    pool = units * unit
    o = oracle.BitmaskOracle(pool, unit)
    held, trace = [], []

    def batch(frees, sizes):
        f = np.array(frees, np.uint64)
        s = np.array(sizes, np.uint64)
        out, st = o.batch(f, s)
        trace.append((f, s, out, st))
        return [int(x) for x in out if x != FAIL]

    for _ in range(8):
        held += batch([], (rng.integers(1, 300, 500) * unit - rng.integers(0, unit, 500)).tolist())
    for _ in range(12):
        held.sort()
        a = int(rng.integers(0, max(1, len(held) - 400)))
        run = held[a:a + int(rng.integers(50, 400))]          # neighbours, freed together
        other = [held[int(i)] for i in rng.choice(len(held), min(len(held), 200), replace=False)]
        picks = run + other
        frees = list(picks)
        frees += [picks[int(i)] for i in rng.integers(0, len(picks), 60)]      # repeats, anywhere
        frees += [h + unit for h in other[:40]] + [h + 3 for h in other[40:60]]  # interior, misaligned
        frees += [pool, pool + unit, 2 * pool]
        frees = [frees[int(i)] for i in rng.permutation(len(frees))]
        freed = set(picks)
        held = [h for h in held if h not in freed]
        held += batch(frees, (rng.integers(1, 300, int(rng.integers(0, 300))) * unit).tolist())
    o2 = oracle.BitmaskOracle(pool, unit)
    for f, s, _, _ in trace:
        o2.batch(f, s)
    _run_bitmask(trace, o2, pool, unit, state_every=2)


@pytest.mark.parametrize("hi", [520, 8192])
def test_bitmask_multi_pool(gpu_lib, hi):
    """Independent pools of different sizes, one CTA each, in one launch;
    objects up to 65 units, and up to 1,024 units (runs across many words)."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import MultiAllocator
    from paper_2405_07079_gb300 import workloads as W

    dev = torch.device("cuda")
    rng = np.random.default_rng(44)
    n = 29
    sizes_a = (rng.integers(64, 20_000, n) * 8).astype(np.uint64)
    m = MultiAllocator(sizes_a, 8, max_total_frees=1 << 16, policy="bitmask")
    orcs = [oracle.BitmaskOracle(int(x), 8) for x in sizes_a]
    clients = [W.TinyRandom(n_ops=10**9, batch=int(rng.integers(1, 200)), p_free=0.45, lo=1, hi=hi,
                            seed=W.BASE_SEED + 700 + i) for i in range(n)]
    for b in range(10):
        fr, sz, exp_o, exp_s = [], [], [], []
        for i in range(n):
            f, s_ = clients[i].next_batch()
            ro, rs = orcs[i].batch(f, s_)
            clients[i].feed(ro)
            fr.append(f); sz.append(s_); exp_o.append(ro); exp_s.append(rs)
        frow = np.concatenate([[0], np.cumsum([x.size for x in fr])]).astype(np.uint32)
        arow = np.concatenate([[0], np.cumsum([x.size for x in sz])]).astype(np.uint32)
        F = np.concatenate(fr).astype(np.uint64)
        S = np.concatenate(sz).astype(np.uint64)
        out = torch.empty(max(1, S.size), dtype=torch.int64, device=dev)
        st = torch.empty(max(1, F.size), dtype=torch.uint8, device=dev)
        m.step(to_dev(frow.view(np.int32), dev), to_dev(F, dev), to_dev(arow.view(np.int32), dev),
               to_dev(S, dev), out, st)
        assert np.array_equal(from_dev(out)[:S.size], np.concatenate(exp_o)), f"batch {b}"
        assert np.array_equal(from_dev(st)[:F.size], np.concatenate(exp_s))
    for i in range(n):
        assert np.array_equal(m.export_state(i), orcs[i].export_state()), i
    m.close()


@pytest.mark.parametrize("policy", ["segfit", "tlsf", "first", "next", "best", "bitmask"])
def test_reset_and_host_pipeline_for_every_policy(gpu_lib, policy):
    """hba_reset returns every policy to its initial state: a trace replayed
    after a reset, through the pipelined host-buffer call, gives the same
    results and state as the first pass through device buffers."""
    import torch

    from paper_2405_07079_gb300 import Allocator, hba_step_host_async
    from paper_2405_07079_gb300 import workloads as W

    wl = W.objects(n_ops=3000, batch=64) if policy == "bitmask" else W.tiny(n_ops=3000)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    with Allocator(wl.arena, wl.min_block, policy=policy) as a:
        cl = wl.make()
        first = []
        while (b := cl.next_batch()) is not None:
            f, s_ = b
            st = torch.empty(f.size, dtype=torch.uint8, device=dev)
            out = a.step(to_dev(f, dev) if f.size else None, to_dev(s_, dev) if s_.size else None, status=st)
            o = from_dev(out) if s_.size else np.zeros(0, np.uint64)
            cl.feed(o)
            first.append((f, s_, o, from_dev(st)))
        state = a.export_state()
        a.reset()
        keep, outs = [], []
        for f, s_, _, _ in first:
            hf = torch.from_numpy(np.ascontiguousarray(f).view(np.int64)).pin_memory()
            hs = torch.from_numpy(np.ascontiguousarray(s_).view(np.int64)).pin_memory()
            ho = torch.empty(max(1, s_.size), dtype=torch.int64).pin_memory()
            hst = torch.empty(max(1, f.size), dtype=torch.uint8).pin_memory()
            keep += [hf, hs, ho, hst]
            hba_step_host_async(a.h, hf.data_ptr() if f.size else 0, f.size, hst.data_ptr() if f.size else 0,
                                hs.data_ptr() if s_.size else 0, s_.size, ho.data_ptr() if s_.size else 0,
                                int(stream.cuda_stream))
            outs.append((ho, hst))
        stream.synchronize()
        for (f, s_, o, st), (ho, hst) in zip(first, outs):
            assert np.array_equal(ho.numpy().view(np.uint64)[:s_.size], o)
            assert np.array_equal(hst.numpy()[:f.size], st)
        assert np.array_equal(a.export_state(), state)
