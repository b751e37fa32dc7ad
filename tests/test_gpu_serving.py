"""The serving loop: requests arriving open loop, all allocator state on the
device.  Its tick log is replayed exactly (the allocator is deterministic
given the batches), through the oracle batch by batch and through the plain
GPU path one request at a time: each request's result is the same in the mix
as alone (integer results: bit-exact)."""
from __future__ import annotations

import numpy as np
import pytest

from _helpers import from_dev, to_dev

pytestmark = pytest.mark.gpu

FAIL = 0xFFFFFFFFFFFFFFFF
REJ = 0xFFFFFFFFFFFFFFFE


def _replay(arr, served, log, arena, mb, one_by_one_gpu=False):
    """Replay the tick log; returns the number of ticks replayed."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator, log_batches

    dev = torch.device("cuda")
    o = oracle.Oracle(arena, mb)
    a = Allocator(arena, mb, threads=256) if one_by_one_gpu else None
    ticks = log_batches(log)
    for t, (fid, aid) in enumerate(ticks):
        frees = served[fid, 0]
        sizes = arr[aid, 1]
        ro, rs = o.batch(frees, sizes)
        assert not rs.any(), f"tick {t}: a logged free was rejected"
        assert np.array_equal(ro, served[aid, 0]), f"tick {t}: mix differs from the oracle"
        if a is not None:
            # alone: every request in its own call, in tick order
            for f in frees:
                st = torch.empty(1, dtype=torch.uint8, device=dev)
                a.step(to_dev(np.array([f], np.uint64), dev), None, status=st)
                assert int(st.cpu()[0]) == 0
            for k, s in enumerate(sizes):
                out = a.step(None, to_dev(np.array([s], np.uint64), dev))
                assert int(from_dev(out)[0]) == int(served[aid[k], 0]), f"tick {t}: alone differs from mix"
    if a is not None:
        assert np.array_equal(a.export_state(), o.export_state())
        a.close()
    return len(ticks)


def test_serving_matches_replay_and_alone(gpu_lib):
    from paper_2405_07079_gb300 import Allocator, serve
    from paper_2405_07079_gb300 import workloads as W

    arena, page = 64 << 20, 16 << 10
    arr = W.serving_arrivals(lam=200_000, seconds=0.03, page=page, max_pages=64, hold_mean_ns=1e6)
    with Allocator(arena, page, threads=256) as a:
        served, log, rep = serve(a, arr, max_batch=512)
        stats = a.stats()
    n = arr.shape[0]
    assert rep["status"] == 0 and rep["arrivals"] == n
    assert rep["admitted"] + rep["rejected"] == n
    assert rep["alloc_ok"] + rep["alloc_fail"] == rep["admitted"]
    assert rep["log_words"] == log.size
    done = served[:, 1] > 0
    assert done.all(), "every request reached a result"
    adm = served[:, 0] != REJ
    ok = adm & (served[:, 0] != FAIL)
    assert int(ok.sum()) == rep["alloc_ok"] == stats["alloc_ok"]
    assert rep["frees"] == int((served[:, 2] > 0).sum()) == stats["free_ok"]
    # timing: results after arrival, frees after the hold
    assert (served[adm, 1] >= arr[adm, 0]).all()
    fr = served[:, 2] > 0
    assert (served[fr, 2] >= served[fr, 1] + arr[fr, 2]).all()
    # continuous batching: several ticks carried several requests
    ticks = _replay(arr, served, log, arena, page, one_by_one_gpu=True)
    assert ticks > 10


def test_serving_rejects_when_the_queue_is_full(gpu_lib):
    from paper_2405_07079_gb300 import Allocator, serve
    from paper_2405_07079_gb300 import workloads as W

    arena, page = 16 << 20, 16 << 10
    arr = W.serving_arrivals(lam=5_000_000, seconds=0.004, page=page, max_pages=256, hold_mean_ns=2e6)
    with Allocator(arena, page, threads=256) as a:
        served, log, rep = serve(a, arr, queue_depth=64, max_batch=256)
    assert rep["rejected"] > 0 and rep["max_queue"] <= 64
    assert int((served[:, 0] == REJ).sum()) == rep["rejected"]
    _replay(arr, served, log, arena, page)
