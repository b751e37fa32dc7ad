"""The serving loop: requests arriving open loop, all allocator state on the
device.  Its tick log is replayed exactly (the allocator is deterministic
given the batches), through the oracle batch by batch and through the plain
GPU path one request at a time: each request's result is the same in the mix
as alone (integer results: bit-exact)."""
from __future__ import annotations

import numpy as np
import pytest

from _helpers import canary_intact, from_dev, to_dev

pytestmark = pytest.mark.gpu

FAIL = 0xFFFFFFFFFFFFFFFF
REJ = 0xFFFFFFFFFFFFFFFE


def _replay(arr, served, log, arena, mb, one_by_one_gpu=False, o=None):
    """Replay the tick log through the oracle ``o`` (a fresh one if None;
    pass the oracle of an earlier run on the same handle to continue from
    its state); returns the number of ticks replayed."""
    import torch

    import oracle
    from paper_2405_07079_gb300 import Allocator, log_batches

    dev = torch.device("cuda")
    o = oracle.Oracle(arena, mb) if o is None else o
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


def _limit_then_normal(arena, page, arr, limited_cfg, expect_status):
    """A run stopped by one of the loop's own limits, then a normal run on
    the same handle: both tick logs replay exactly through one oracle, and
    the device's final state equals the oracle's."""
    import oracle
    from paper_2405_07079_gb300 import Allocator, HbaError, serve
    from paper_2405_07079_gb300 import workloads as W

    o = oracle.Oracle(arena, page)
    with Allocator(arena, page, threads=256) as a:
        if expect_status == 2:
            with pytest.raises(HbaError) as ei:
                serve(a, arr, **limited_cfg)
            assert ei.value.code == 5  # HBA_ERR_STATE
            served, log, rep = ei.value.served, ei.value.log, ei.value.report
        else:
            served, log, rep = serve(a, arr, **limited_cfg)
        assert rep["status"] == expect_status, rep
        assert rep["arrivals"] <= arr.shape[0]
        _replay(arr, served, log, arena, page, o=o)
        arr2 = W.serving_arrivals(lam=100_000, seconds=0.01, page=page, max_pages=32, hold_mean_ns=1e6, seed=99)
        served2, log2, rep2 = serve(a, arr2, max_batch=512)
        assert rep2["status"] == 0 and rep2["arrivals"] == arr2.shape[0]
        _replay(arr2, served2, log2, arena, page, o=o)
        assert np.array_equal(a.export_state(), o.export_state())
    return rep


def test_serving_time_limit_stops_the_run(gpu_lib):
    """time_limit_ns shorter than the arrivals: the loop stops at the first
    tick past the limit with status 1 (time limit), having taken only part of
    the arrivals; the handle stays usable."""
    from paper_2405_07079_gb300 import workloads as W

    arena, page = 64 << 20, 16 << 10
    arr = W.serving_arrivals(lam=200_000, seconds=0.05, page=page, max_pages=64, hold_mean_ns=1e6)
    rep = _limit_then_normal(arena, page, arr, dict(max_batch=512, time_limit_ns=2_000_000), expect_status=1)
    assert rep["arrivals"] < arr.shape[0] and rep["elapsed_ns"] >= 2_000_000


def test_serving_tick_limit_stops_the_run(gpu_lib):
    """max_ticks = 3: the loop runs exactly three ticks, reports status 3."""
    from paper_2405_07079_gb300 import workloads as W

    arena, page = 64 << 20, 16 << 10
    arr = W.serving_arrivals(lam=200_000, seconds=0.05, page=page, max_pages=64, hold_mean_ns=1e6)
    rep = _limit_then_normal(arena, page, arr, dict(max_batch=512, max_ticks=3), expect_status=3)
    assert rep["ticks"] == 3


def test_serving_wheel_full_is_an_error(gpu_lib):
    """Holds longer than the free-timing wheel spans (4,096 buckets of 1 us
    against holds of about 10 ms): the loop stops with status 2 and the call
    returns HBA_ERR_STATE, with the report, results and log of the ticks
    that ran; the handle stays usable."""
    from paper_2405_07079_gb300 import workloads as W

    arena, page = 64 << 20, 16 << 10
    arr = W.serving_arrivals(lam=200_000, seconds=0.02, page=page, max_pages=64, hold_mean_ns=1e7)
    rep = _limit_then_normal(arena, page, arr, dict(max_batch=512, bucket_ns=1000), expect_status=2)
    assert rep["ticks"] >= 1


def test_serving_at_the_80GiB_page_shape(gpu_lib):
    """The 80 GiB arena of 16 KiB pages (5,242,880 pages), U{1..512}-page
    requests held Exp(20 ms), at 1 M requests/s for 50 ms: every tick
    replays exactly through the oracle, and a real 80 GiB arena filled with
    the canary byte is left untouched."""
    import torch

    from paper_2405_07079_gb300 import Allocator, serve
    from paper_2405_07079_gb300 import workloads as W

    arena, page = 80 << 30, 16 << 10
    arr = W.serving_arrivals(lam=1_000_000, seconds=0.05, page=page, max_pages=512, hold_mean_ns=20e6)
    guard = torch.full((arena,), 0xA5, dtype=torch.uint8, device="cuda")
    with Allocator(arena, page, threads=256) as a:
        served, log, rep = serve(a, arr)
    assert rep["status"] == 0 and rep["arrivals"] == arr.shape[0]
    assert rep["alloc_ok"] > 10_000
    ticks = _replay(arr, served, log, arena, page)
    assert ticks > 10
    torch.cuda.synchronize()
    assert canary_intact(guard), "the managed arena was written"
    del guard
