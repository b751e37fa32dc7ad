"""CPU oracles of the allocators of the paper: segregated fit (§5.1,
Algorithms 4 and 5, the evaluated one), two-level segregated fit (§5.2), the
sequential fits on address-sorted lists (§3.1, §4) and the bitmask pool
(§3.2).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
library in ``paper_2405_07079_gb300`` never imports it, and the two share no
code: the only module both sides use is the seeded request generator
(``paper_2405_07079_gb300.workloads``), which holds none of the allocator's
arithmetic.

Each policy has two independent statements that pin each other:

* ``Oracle`` -- ``segfit_oracle.c``: the paper's own structures (hash table
  keyed by address, doubly linked LIFO free lists per power-of-two class, a
  64-bit availability bitmap), Algorithms 4 and 5 step by step; with
  ``policy="tlsf"`` the same algorithms with the two-tier lookup of §5.2.
  ``space()`` reports the largest free block and the extent (Fig. 4).
* ``interval_ref.IntervalAllocator`` -- a brute-force restatement over a
  sorted list of intervals with push stamps (both policies), used on tiny
  arenas to pin the first one (see that module's header).
* ``HalOracle`` -- ``hal_oracle.c``: first, next and best fit on sorted free
  and used lists with partial deallocation; pinned by
  ``fits_ref.GranuleFits``, a granule -> owner map.
* ``BitmaskOracle`` -- ``bitmask_oracle.c``: the bitmask pool; pinned by
  ``fits_ref.BlockListPool``, a list of in-use intervals.

Parity against the paper's experiment (Fig. 3 / Fig. 4 of §6) is unpinned:
the paper prints no data for those figures.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "segfit_oracle.c")
_HAL_SRC = os.path.join(_HERE, "hal_oracle.c")
_BM_SRC = os.path.join(_HERE, "bitmask_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsegfit_oracle.so")
_lock = threading.Lock()
_lib = None

FAIL = np.uint64(0xFFFFFFFFFFFFFFFF)


def build(force: bool = False) -> str:
    """Compile ``segfit_oracle.c`` into ``_build/libsegfit_oracle.so`` (gcc)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(map(os.path.getmtime, (_SRC, _HAL_SRC, _BM_SRC))))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, _HAL_SRC, _BM_SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
            lib.orc_create.restype = vp
            lib.orc_create.argtypes = [u64, u64]
            lib.orc_create_policy.restype = vp
            lib.orc_create_policy.argtypes = [u64, u64, ctypes.c_int]
            lib.orc_destroy.argtypes = [vp]
            lib.orc_arena.restype = u64
            lib.orc_arena.argtypes = [vp]
            lib.orc_malloc.restype = u64
            lib.orc_malloc.argtypes = [vp, u64]
            lib.orc_free.restype = ctypes.c_int
            lib.orc_free.argtypes = [vp, u64]
            lib.orc_batch.argtypes = [vp, vp, u32, vp, vp, u32, vp]
            lib.orc_export.restype = ctypes.c_size_t
            lib.orc_export.argtypes = [vp, vp, ctypes.c_size_t]
            lib.orc_stats.argtypes = [vp, vp]
            lib.orc_space.argtypes = [vp, vp]
            lib.hal_create.restype = vp
            lib.hal_create.argtypes = [u64, u64, ctypes.c_int]
            lib.hal_destroy.argtypes = [vp]
            lib.hal_malloc.restype = u64
            lib.hal_malloc.argtypes = [vp, u64]
            lib.hal_free.restype = ctypes.c_int
            lib.hal_free.argtypes = [vp, u64]
            lib.hal_batch.argtypes = [vp, vp, u32, vp, vp, u32, vp]
            lib.hal_export.restype = ctypes.c_size_t
            lib.hal_export.argtypes = [vp, vp, ctypes.c_size_t]
            lib.hal_stats.argtypes = [vp, vp]
            lib.bm_create.restype = vp
            lib.bm_create.argtypes = [u64, u64]
            lib.bm_destroy.argtypes = [vp]
            lib.bm_malloc.restype = u64
            lib.bm_malloc.argtypes = [vp, u64]
            lib.bm_free.restype = ctypes.c_int
            lib.bm_free.argtypes = [vp, u64]
            lib.bm_batch.argtypes = [vp, vp, u32, vp, vp, u32, vp]
            lib.bm_export.restype = ctypes.c_size_t
            lib.bm_export.argtypes = [vp, vp, ctypes.c_size_t]
            lib.bm_stats.argtypes = [vp, vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


POLICIES = {"segfit": 0, "tlsf": 1}


class Oracle:
    """One arena managed by the sequential oracle: segregated fit (§5.1),
    or with ``policy="tlsf"`` two-level segregated fit (§5.2)."""

    STAT_KEYS = ("alloc_ok", "alloc_fail", "free_ok", "free_fail", "used_bytes",
                 "used_blocks", "blocks", "requested_bytes", "bitmask")

    def __init__(self, arena_bytes: int, min_block: int, policy: str = "segfit"):
        self._lib = _load()
        self.policy = policy
        self._h = self._lib.orc_create_policy(int(arena_bytes), int(min_block), POLICIES[policy])
        if not self._h:
            raise ValueError("invalid arena_bytes/min_block")
        self.arena = int(self._lib.orc_arena(self._h))
        self.min_block = int(min_block)

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def malloc(self, size: int) -> int:
        return int(self._lib.orc_malloc(self._h, int(size)))

    def free(self, addr: int) -> int:
        return int(self._lib.orc_free(self._h, int(addr)))

    def batch(self, frees, sizes):
        """Apply one batch (frees in index order, then allocations).

        Returns ``(out_offsets uint64[na], free_status uint8[nf])``."""
        f = np.ascontiguousarray(frees, dtype=np.uint64)
        s = np.ascontiguousarray(sizes, dtype=np.uint64)
        out = np.empty(s.size, dtype=np.uint64)
        st = np.empty(f.size, dtype=np.uint8)
        self._lib.orc_batch(self._h, _ptr(f), f.size, _ptr(st), _ptr(s), s.size, _ptr(out))
        return out, st

    def export_state(self) -> np.ndarray:
        n = self._lib.orc_export(self._h, None, 0)
        buf = np.empty(n, dtype=np.uint64)
        self._lib.orc_export(self._h, buf.ctypes.data, n)
        return buf

    def stats(self) -> dict:
        buf = np.zeros(9, dtype=np.uint64)
        self._lib.orc_stats(self._h, buf.ctypes.data)
        return {k: int(v) for k, v in zip(self.STAT_KEYS, buf)}

    def space(self) -> dict:
        """Largest free block and extent (end of the highest in-use block,
        0 when none): the memory-usage view of §6, Fig. 4."""
        buf = np.zeros(2, dtype=np.uint64)
        self._lib.orc_space(self._h, buf.ctypes.data)
        return {"largest_free": int(buf[0]), "extent": int(buf[1])}


FITS = {"first": 0, "next": 1, "best": 2}


class HalOracle:
    """One arena managed by a sequential fit on address-sorted free and used
    lists (§3.1 Algorithms 1 and 2, §4 Algorithm 3 and its first-fit and
    next-fit variants), with partial deallocation."""

    STAT_KEYS = ("alloc_ok", "alloc_fail", "free_ok", "free_fail", "used_bytes", "used_blocks", "blocks",
                 "requested_bytes", "largest_free", "extent")

    def __init__(self, arena_bytes: int, min_block: int, fit: str = "first"):
        self._lib = _load()
        self.fit = fit
        self._h = self._lib.hal_create(int(arena_bytes), int(min_block), FITS[fit])
        if not self._h:
            raise ValueError("invalid arena_bytes/min_block/fit")
        self.min_block = int(min_block)

    def close(self):
        if self._h:
            self._lib.hal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def malloc(self, size: int) -> int:
        return int(self._lib.hal_malloc(self._h, int(size)))

    def free(self, addr: int) -> int:
        return int(self._lib.hal_free(self._h, int(addr)))

    def batch(self, frees, sizes):
        f = np.ascontiguousarray(frees, dtype=np.uint64)
        s = np.ascontiguousarray(sizes, dtype=np.uint64)
        out = np.empty(s.size, dtype=np.uint64)
        st = np.empty(f.size, dtype=np.uint8)
        self._lib.hal_batch(self._h, _ptr(f), f.size, _ptr(st), _ptr(s), s.size, _ptr(out))
        return out, st

    def export_state(self) -> np.ndarray:
        n = self._lib.hal_export(self._h, None, 0)
        buf = np.empty(n, dtype=np.uint64)
        self._lib.hal_export(self._h, buf.ctypes.data, n)
        return buf

    def stats(self) -> dict:
        buf = np.zeros(10, dtype=np.uint64)
        self._lib.hal_stats(self._h, buf.ctypes.data)
        return {k: int(v) for k, v in zip(self.STAT_KEYS, buf)}


class BitmaskOracle:
    """A bitmask pool (§3.2): one free bit per unit of ``unit`` bytes, runs
    found by next fit, a second out-of-band bitmap marking block starts."""

    STAT_KEYS = HalOracle.STAT_KEYS

    def __init__(self, pool_bytes: int, unit: int):
        self._lib = _load()
        self._h = self._lib.bm_create(int(pool_bytes), int(unit))
        if not self._h:
            raise ValueError("invalid pool_bytes/unit")
        self.unit = int(unit)

    def close(self):
        if self._h:
            self._lib.bm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def malloc(self, size: int) -> int:
        return int(self._lib.bm_malloc(self._h, int(size)))

    def free(self, addr: int) -> int:
        return int(self._lib.bm_free(self._h, int(addr)))

    def batch(self, frees, sizes):
        f = np.ascontiguousarray(frees, dtype=np.uint64)
        s = np.ascontiguousarray(sizes, dtype=np.uint64)
        out = np.empty(s.size, dtype=np.uint64)
        st = np.empty(f.size, dtype=np.uint8)
        self._lib.bm_batch(self._h, _ptr(f), f.size, _ptr(st), _ptr(s), s.size, _ptr(out))
        return out, st

    def export_state(self) -> np.ndarray:
        n = self._lib.bm_export(self._h, None, 0)
        buf = np.empty(n, dtype=np.uint64)
        self._lib.bm_export(self._h, buf.ctypes.data, n)
        return buf

    def stats(self) -> dict:
        buf = np.zeros(10, dtype=np.uint64)
        self._lib.bm_stats(self._h, buf.ctypes.data)
        return {k: int(v) for k, v in zip(self.STAT_KEYS, buf)}


def decode_hal_state(words) -> dict:
    """Split a sequential-fit canonical state (H10) into its parts."""
    w = [int(x) for x in words]
    arena, mb, nf = w[0], w[1], w[2]
    free = [(w[3 + 2 * i], w[4 + 2 * i]) for i in range(nf)]
    i = 3 + 2 * nf
    nu = w[i]
    used = [(w[i + 1 + 2 * k], w[i + 2 + 2 * k]) for k in range(nu)]
    i += 1 + 2 * nu
    assert i + 1 == len(w), "trailing words in canonical state"
    return {"arena": arena, "min_block": mb, "free": free, "used": used, "rover": w[i]}


def decode_state(words, policy: str = "segfit") -> dict:
    """Split a canonical state (R11; T4 for TLSF) into its parts for
    readable assertions."""
    w = [int(x) for x in words]
    arena, min_block, nblocks = w[0], w[1], w[2]
    blocks = []
    i = 3
    a = 0
    while a < arena:
        off = w[i]
        if off == 0xFFFFFFFFFFFFFFFF:
            raise AssertionError("blocks do not tile the arena")
        sz = w[i + 1] & ((1 << 63) - 1)
        blocks.append((off, sz, bool(w[i + 1] >> 63)))
        a = off + sz
        i += 2
    bins = []
    for _ in range(64 if policy == "segfit" else 64 * 16):
        cnt = w[i]
        bins.append(w[i + 1:i + 1 + cnt])
        i += 1 + cnt
    bitmask = w[i]
    i += 1
    slmask = []
    if policy == "tlsf":
        slmask = w[i:i + 64]
        i += 64
    assert i == len(w), "trailing words in canonical state"
    return {"arena": arena, "min_block": min_block, "nblocks": nblocks,
            "blocks": blocks, "bins": bins, "bitmask": bitmask, "slmask": slmask}
