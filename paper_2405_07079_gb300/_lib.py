"""ctypes loader of ``_build/libhba.so`` (the C ABI declared in include/hba.h).

There is no fallback: if the library has not been built, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

_lock = threading.Lock()
_lib = None

STATUS = {0: "HBA_OK", 1: "HBA_ERR_INVALID_ARGUMENT", 2: "HBA_ERR_OUT_OF_MEMORY", 3: "HBA_ERR_CUDA",
          4: "HBA_ERR_TIMEOUT", 5: "HBA_ERR_STATE"}

# Every symbol include/hba.h declares, with (restype, argtypes).
u64, u32, i32, vp, sz = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
SIGNATURES = {
    "hba_create": (i32, [u64, u64, i32, vp]),
    "hba_create_ex": (i32, [u64, u64, i32, u32, vp]),
    "hba_destroy": (i32, [vp]),
    "hba_alloc_batch": (i32, [vp, vp, u32, vp, vp]),
    "hba_free_batch": (i32, [vp, vp, u32, vp]),
    "hba_free_batch_ex": (i32, [vp, vp, u32, vp, vp]),
    "hba_step": (i32, [vp, vp, u32, vp, vp, u32, vp, vp]),
    "hba_step_host": (i32, [vp, vp, u32, vp, vp, u32, vp, vp]),
    "hba_step_host_async": (i32, [vp, vp, u32, vp, vp, u32, vp, vp]),
    "hba_step_static": (i32, [vp, vp, u32, vp, vp, u32, vp, vp]),
    "hba_reset": (i32, [vp, vp]),
    "hba_stats": (i32, [vp, vp]),
    "hba_export_state": (i32, [vp, u32, vp, sz, vp]),
    "hba_multi_create": (i32, [u32, vp, u64, i32, u32, vp]),
    "hba_multi_step": (i32, [vp, vp, vp, u32, vp, vp, u32, vp, vp, vp]),
    "hba_multi_create_ex": (i32, [u32, vp, u64, i32, u32, u32, vp]),
    "hba_multi_step_host_async": (i32, [vp, vp, vp, u32, vp, vp, u32, vp, vp, vp]),
    "hba_set_shape": (i32, [vp, u32, u32, u32]),
    "hba_serve_run": (i32, [vp, vp, u64, vp, vp, u64, vp, vp, vp]),
    "hba_version": (ctypes.c_char_p, []),
    "hba_launch_count": (i32, [vp, vp]),
}


class HbaError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {STATUS.get(code, code)}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "alloc_ok", "alloc_fail", "free_ok", "free_fail", "used_bytes", "used_blocks", "blocks",
        "requested_bytes", "free_bytes", "largest_free", "bitmask", "arena_bytes", "extent_bytes")] + [
        ("n_arenas", ctypes.c_uint32), ("device_error", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class ServeConfig(ctypes.Structure):
    _fields_ = [("queue_depth", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("bucket_ns", ctypes.c_uint64),
                ("time_limit_ns", ctypes.c_uint64), ("max_ticks", ctypes.c_uint64)]


class ServeReport(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "arrivals", "admitted", "rejected", "alloc_ok", "alloc_fail", "frees", "ticks", "idle_ticks",
        "max_queue", "elapsed_ns", "status", "log_words")]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


def load(path: str = LIB):
    """Load the built library; raises OSError if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise OSError(f"{path} is not built; run paper_2405_07079_gb300.build.build_library()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype, f.argtypes = res, args
            _lib = lib
    return _lib


def check(fn: str, code: int):
    if code != 0:
        raise HbaError(fn, code)
