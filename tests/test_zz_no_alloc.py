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


def test_static_scratch_matches_hba_step(gpu_lib):
    import torch

    from paper_2405_07079_gb300 import Allocator, hba_step, hba_step_static
    from paper_2405_07079_gb300 import workloads as W
    from paper_2405_07079_gb300.hba import _ptr

    dev = torch.device("cuda")
    # batches of 4,096 requests with small sizes: about 2,000 frees per batch,
    # up to the static maximum of 4,096
    wl = W.Workload("life-256MiB", 1 << 28, 512,
                    lambda: W.Lifetimes(n_ops=120_000, batch=4096, mean_life=150, scale=1 / 256, min_size=512))
    trace, _ = oracle_trace(wl)
    assert max(f.size for f, _, _, _ in trace) > 2000
    ref = Allocator(wl.arena, wl.min_block)                  # handle scratch (hba_step)
    stat = Allocator(wl.arena, wl.min_block, max_batch=1)    # no room: static scratch only
    try:
        for b, (f, s, _, _) in enumerate(trace):
            df, ds = to_dev(f, dev), to_dev(s, dev)
            o1 = torch.empty(s.size, dtype=torch.int64, device=dev)
            o2 = torch.empty(s.size, dtype=torch.int64, device=dev)
            s1 = torch.empty(f.size, dtype=torch.uint8, device=dev)
            s2 = torch.empty(f.size, dtype=torch.uint8, device=dev)
            stream = int(torch.cuda.current_stream().cuda_stream)
            hba_step(ref.h, _ptr(df), f.size, _ptr(s1), _ptr(ds), s.size, _ptr(o1), stream)
            hba_step_static(stat.h, _ptr(df), f.size, _ptr(s2), _ptr(ds), s.size, _ptr(o2), stream)
            assert np.array_equal(from_dev(o1), from_dev(o2)), f"batch {b}: offsets differ"
            assert np.array_equal(from_dev(s1), from_dev(s2)), f"batch {b}: free statuses differ"
            if b < 3 or b % 8 == 0:
                assert np.array_equal(ref.export_state(), stat.export_state()), f"batch {b}: state"
        assert np.array_equal(ref.export_state(), stat.export_state())
        assert ref.stats() == stat.stats()
    finally:
        ref.close()
        stat.close()


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
