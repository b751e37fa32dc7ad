"""The CUDA runtime's allocators on the same operations, for comparison.

The paper (§6) compares segregated fit with ``cudaMalloc``/``cudaFree`` on
one operation order.  ``trace_ops`` turns a recorded batched trace (requests
plus this allocator's results) into that order -- each batch's applied frees
in index order, then its served allocations -- and ``replay`` runs it through
``cudaMalloc``/``cudaFree`` (mode 0) or ``cudaMallocAsync``/``cudaFreeAsync``
on a stream with the default pool (mode 1), timing every call on the host.
Failed allocations and rejected frees are not replayed: the CUDA allocators
draw on the whole device, so they would succeed and never be freed.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_BUILD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
REPLAY_LIB = os.path.join(_BUILD, "libcuda_replay.so")
FAIL = np.uint64(0xFFFFFFFFFFFFFFFF)
MODES = {"cudaMalloc": 0, "cudaMallocAsync": 1}

_lib = None


def trace_ops(batches) -> np.ndarray:
    """``batches``: iterable of ``(frees, status, sizes, out)`` numpy arrays
    (uint64 offsets, uint8 free status with 0 = applied, uint64 sizes, uint64
    results with ``FAIL`` for a failed allocation).  Returns the int64 op
    list: ``size >= 0`` is a malloc filling the next slot, ``-(k + 1)`` frees
    slot k."""
    live = {}
    ops = []
    nslot = 0
    for frees, status, sizes, out in batches:
        for off, st in zip(frees.tolist(), status.tolist()):
            if st == 0:
                ops.append(-(live.pop(off) + 1))
        for sz, off in zip(sizes.tolist(), out.tolist()):
            if off != int(FAIL):
                if off in live:
                    raise ValueError(f"offset {off} served twice without a free")
                live[off] = nslot
                nslot += 1
                ops.append(int(sz))
    return np.asarray(ops, dtype=np.int64)


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(REPLAY_LIB):
            raise RuntimeError(f"{REPLAY_LIB} is missing: build the package first")
        lib = ctypes.CDLL(REPLAY_LIB)
        lib.car_replay.restype = ctypes.c_int64
        lib.car_replay.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def replay(ops: np.ndarray, mode: str, stream: int = 0) -> dict:
    """Run ``ops`` through the CUDA allocator ``mode`` ("cudaMalloc" or
    "cudaMallocAsync").  Returns ops/s over the whole replay (final
    synchronisation included) and per-call host latency percentiles."""
    ops = np.ascontiguousarray(ops, dtype=np.int64)
    lat = np.zeros(ops.size, dtype=np.int64)
    total = _load().car_replay(ops.ctypes.data, ops.size, MODES[mode], lat.ctypes.data, ctypes.c_void_p(stream))
    if total < 0:
        raise RuntimeError(f"{mode} replay failed with code {total}")
    n = int(ops.size)
    srt = np.sort(lat)
    pct = (lambda q: float(srt[min(n - 1, int(q * n))]) / 1e3) if n else (lambda q: 0.0)
    return {"value": n / (total / 1e9) if total else 0.0, "unit": "ops/s", "ops": n,
            "mallocs": int((ops >= 0).sum()), "frees": int((ops < 0).sum()),
            "p50_us": pct(0.50), "p99_us": pct(0.99), "total_ms": total / 1e6}
