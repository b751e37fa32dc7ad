"""hba_step_static: the batch entry point that allocates nothing.

Callers that cannot allocate device memory when they run batches (many small
handles under a fixed device-memory budget, or memory reserved up front by
another pool) create their handles with max_batch = 1 and run batches through
hba_step_static, whose kernels take their scratch from one static device
array in the library.  This file checks, through the C ABI, that it returns
exactly what hba_step returns on the same inputs (the allocator's results are
integers: the comparison is bit-exact), batch after batch, and that it
rejects batches with more frees than the static array holds.  It is collected
last so that a stop at the first failure has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

from _helpers import from_dev, oracle_trace, to_dev

pytestmark = pytest.mark.gpu


def _compare_static(trace, arena, min_block, threads=None, ctas=0, smem_bytes=0):
    """Replay an oracle trace through hba_step (a handle with its own
    scratch) and hba_step_static (a handle with none) on the same inputs:
    offsets and free statuses equal each other and the oracle's, batch by
    batch; states and counters equal at the end."""
    import torch

    from paper_2405_07079_gb300 import Allocator, hba_step, hba_step_static
    from paper_2405_07079_gb300.hba import _ptr

    dev = torch.device("cuda")
    ref = Allocator(arena, min_block, threads=threads, ctas=ctas, smem_bytes=smem_bytes)  # handle scratch
    stat = Allocator(arena, min_block, max_batch=1, threads=threads, ctas=ctas, smem_bytes=smem_bytes)  # none
    try:
        for b, (f, s, out, st) in enumerate(trace):
            df, ds = to_dev(f, dev), to_dev(s, dev)
            o1 = torch.empty(s.size, dtype=torch.int64, device=dev)
            o2 = torch.empty(s.size, dtype=torch.int64, device=dev)
            s1 = torch.empty(f.size, dtype=torch.uint8, device=dev)
            s2 = torch.empty(f.size, dtype=torch.uint8, device=dev)
            stream = int(torch.cuda.current_stream().cuda_stream)
            hba_step(ref.h, _ptr(df), f.size, _ptr(s1), _ptr(ds), s.size, _ptr(o1), stream)
            hba_step_static(stat.h, _ptr(df), f.size, _ptr(s2), _ptr(ds), s.size, _ptr(o2), stream)
            g1, g2 = from_dev(o1), from_dev(o2)
            assert np.array_equal(g1, g2), f"batch {b}: offsets differ"
            assert np.array_equal(g2, out), f"batch {b}: offsets differ from the oracle"
            assert np.array_equal(from_dev(s1), from_dev(s2)), f"batch {b}: free statuses differ"
            assert np.array_equal(from_dev(s2), st), f"batch {b}: free statuses differ from the oracle"
            if b < 3 or b % 8 == 0:
                assert np.array_equal(ref.export_state(), stat.export_state()), f"batch {b}: state"
        assert np.array_equal(ref.export_state(), stat.export_state())
        assert ref.stats() == stat.stats()
        return stat.export_state()
    finally:
        ref.close()
        stat.close()


def test_static_scratch_matches_hba_step(gpu_lib):
    from paper_2405_07079_gb300 import workloads as W

    # batches of 4,096 requests with small sizes: about 2,000 frees per batch
    wl = W.Workload("life-256MiB", 1 << 28, 512,
                    lambda: W.Lifetimes(n_ops=120_000, batch=4096, mean_life=150, scale=1 / 256, min_size=512))
    trace, o = oracle_trace(wl)
    assert max(f.size for f, _, _, _ in trace) > 2000
    assert np.array_equal(_compare_static(trace, wl.arena, wl.min_block), o.export_state())


def test_static_scratch_full_free_batches_global_phase(gpu_lib):
    """Batches of up to the static maximum of valid frees (4,096), with the
    engine's shared memory cut to its minimum so that the free phase works on
    the static array's global working area, and with a two-CTA cluster that
    gathers the frees' records: the largest use of the array."""
    import oracle
    from paper_2405_07079_gb300 import HBA_STATIC_MAX_FREES

    arena, mb = 1 << 30, 256
    o = oracle.Oracle(arena, mb)
    rng = np.random.default_rng(77)
    trace, held = [], []
    for b in range(8):
        nf = min(len(held), HBA_STATIC_MAX_FREES - (b % 2) * 96)
        idx = rng.permutation(len(held))[:nf]
        f = np.array([held[i] for i in idx], np.uint64)
        keep = np.ones(len(held), bool)
        keep[idx] = False
        held = [h for h, k in zip(held, keep) if k]
        s = (rng.integers(1, 256, HBA_STATIC_MAX_FREES) * mb).astype(np.uint64)
        out, st = o.batch(f, s)
        assert (st == 0).all()
        trace.append((f, s, out, st))
        held += [int(x) for x in out if x != np.uint64(0xFFFFFFFFFFFFFFFF)]
    assert max(t[0].size for t in trace) == HBA_STATIC_MAX_FREES
    for shape in ((1024, 2, 1), (1024, 0, 1)):
        assert np.array_equal(_compare_static(trace, arena, mb, *shape), o.export_state())


def test_static_scratch_rejects_oversized_batches(gpu_lib):
    import torch

    from paper_2405_07079_gb300 import HBA_STATIC_MAX_FREES, Allocator, HbaError, hba_step_static
    from paper_2405_07079_gb300.hba import _ptr

    dev = torch.device("cuda")
    with Allocator(1 << 24, 256, max_batch=1) as a:
        frees = torch.zeros(HBA_STATIC_MAX_FREES + 1, dtype=torch.int64, device=dev)
        with pytest.raises(HbaError) as ei:
            hba_step_static(a.h, _ptr(frees), frees.numel(), 0, 0, 0, 0, 0)
        assert ei.value.code == 1  # HBA_ERR_INVALID_ARGUMENT
        # the largest allowed batch still runs, and the handle is unchanged by the rejection
        ok = frees[:HBA_STATIC_MAX_FREES]
        st = torch.empty(ok.numel(), dtype=torch.uint8, device=dev)
        hba_step_static(a.h, _ptr(ok), ok.numel(), _ptr(st), 0, 0, 0, 0)
        torch.cuda.synchronize()
        assert bool((st == 1).all())           # nothing was allocated: every free is rejected
        assert a.stats()["free_fail"] == HBA_STATIC_MAX_FREES
