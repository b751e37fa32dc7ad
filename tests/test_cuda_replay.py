"""The comparison replay through the CUDA runtime's allocators: the op list
built from a batched trace, the replay library's export and argument checks
(CPU), and one short replay per mode on the GPU."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from _helpers import FAIL, oracle_trace


def _u64(*v):
    return np.array(v, dtype=np.uint64)


def test_trace_ops_by_hand():
    from paper_2405_07079_gb300.cuda_replay import trace_ops

    batches = [
        # allocations: two served, one failed
        (_u64(), np.zeros(0, np.uint8), _u64(4096, 1 << 40, 512), _u64(0, FAIL, 4096)),
        # free offset 0 (applied), a rejected free, then a new allocation at 0
        (_u64(0, 77), np.array([0, 1], np.uint8), _u64(256), _u64(0)),
        # free both live blocks (offset 4096 was slot 1, offset 0 is slot 2 now)
        (_u64(4096, 0), np.array([0, 0], np.uint8), _u64(), _u64()),
    ]
    assert trace_ops(batches).tolist() == [4096, 512, -1, 256, -2, -3]


def test_trace_ops_on_an_oracle_trace_is_well_formed():
    """Every free names a slot that a malloc filled and nothing freed since;
    the counts equal the oracle's served allocations and applied frees."""
    from paper_2405_07079_gb300 import workloads
    from paper_2405_07079_gb300.cuda_replay import trace_ops

    trace, _ = oracle_trace(workloads.tiny(n_ops=3000))
    ops = trace_ops((f, st, s, o) for f, s, o, st in trace)
    live, nslot = set(), 0
    for op in ops.tolist():
        if op >= 0:
            live.add(nslot); nslot += 1
        else:
            assert -op - 1 in live
            live.remove(-op - 1)
    assert nslot == sum(int((o != FAIL).sum()) for _, _, o, _ in trace)
    assert int((ops < 0).sum()) == sum(int((st == 0).sum()) for *_, st in trace)


def test_replay_library_exports_and_rejects_bad_arguments():
    from paper_2405_07079_gb300.build import REPLAY_LIB, build_library

    build_library()
    lib = ctypes.CDLL(REPLAY_LIB)
    lib.car_replay.restype = ctypes.c_int64
    lib.car_replay.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    ops = np.array([64], dtype=np.int64)
    assert lib.car_replay(ops.ctypes.data, 1, 7, None, None) == -1      # unknown mode
    assert lib.car_replay(None, 3, 0, None, None) == -1                 # no op list
    assert lib.car_replay(ops.ctypes.data, -1, 0, None, None) == -1     # negative count


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["cudaMalloc", "cudaMallocAsync"])
def test_replay_runs_on_the_gpu(gpu_lib, mode):
    import torch

    from paper_2405_07079_gb300 import workloads
    from paper_2405_07079_gb300.cuda_replay import replay, trace_ops

    trace, _ = oracle_trace(workloads.tiny(n_ops=2000))
    ops = trace_ops((f, st, s, o) for f, s, o, st in trace)
    r = replay(ops, mode, int(torch.cuda.current_stream().cuda_stream))
    assert r["ops"] == ops.size and r["value"] > 0 and r["p99_us"] >= r["p50_us"] >= 0
