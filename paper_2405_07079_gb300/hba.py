"""Thin Python binding of the C ABI (include/hba.h).

The functions ``hba_*`` mirror the C entry points one to one (argument
marshalling only: raw device pointers are ints, streams are ``cudaStream_t``
ints).  ``Allocator`` and ``MultiAllocator`` wrap them for torch tensors:
PyTorch provides device memory and streams, every step of the allocator runs
in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import HbaError, ServeConfig, ServeReport, Stats, check, load

HBA_FAIL = 0xFFFFFFFFFFFFFFFF
HBA_POLICY_SEGFIT = 0
HBA_POLICY_TLSF = 1
HBA_POLICY_FIRST_FIT, HBA_POLICY_NEXT_FIT, HBA_POLICY_BEST_FIT = 2, 3, 4
HBA_POLICY_BITMASK = 5
POLICIES = {"segfit": HBA_POLICY_SEGFIT, "tlsf": HBA_POLICY_TLSF, "first": HBA_POLICY_FIRST_FIT,
            "next": HBA_POLICY_NEXT_FIT, "best": HBA_POLICY_BEST_FIT, "bitmask": HBA_POLICY_BITMASK}


def _lib():
    return load()


# ---- one-to-one wrappers ------------------------------------------------------

def hba_create(arena_bytes: int, min_block: int, policy: int = HBA_POLICY_SEGFIT, max_batch: int | None = None) -> int:
    h = ctypes.c_void_p()
    if max_batch is None:
        check("hba_create", _lib().hba_create(arena_bytes, min_block, policy, ctypes.byref(h)))
    else:
        check("hba_create_ex", _lib().hba_create_ex(arena_bytes, min_block, policy, max_batch, ctypes.byref(h)))
    return h.value


def hba_destroy(h: int) -> None:
    check("hba_destroy", _lib().hba_destroy(h))


def hba_alloc_batch(h: int, d_sizes: int, n: int, d_out: int, stream: int = 0) -> None:
    check("hba_alloc_batch", _lib().hba_alloc_batch(h, d_sizes, n, d_out, stream))


def hba_free_batch(h: int, d_offsets: int, n: int, stream: int = 0) -> None:
    check("hba_free_batch", _lib().hba_free_batch(h, d_offsets, n, stream))


def hba_free_batch_ex(h: int, d_offsets: int, n: int, d_status: int, stream: int = 0) -> None:
    check("hba_free_batch_ex", _lib().hba_free_batch_ex(h, d_offsets, n, d_status, stream))


def hba_step(h: int, d_frees: int, nf: int, d_status: int, d_sizes: int, na: int, d_out: int, stream: int = 0) -> None:
    check("hba_step", _lib().hba_step(h, d_frees, nf, d_status, d_sizes, na, d_out, stream))


def hba_step_host(h: int, h_frees: int, nf: int, h_status: int, h_sizes: int, na: int, h_out: int, stream: int = 0) -> None:
    check("hba_step_host", _lib().hba_step_host(h, h_frees, nf, h_status, h_sizes, na, h_out, stream))


def hba_step_host_async(h: int, h_frees: int, nf: int, h_status: int, h_sizes: int, na: int, h_out: int,
                        stream: int = 0) -> None:
    check("hba_step_host_async",
          _lib().hba_step_host_async(h, h_frees, nf, h_status, h_sizes, na, h_out, stream))


HBA_STATIC_MAX_FREES = 4096


def hba_step_static(h: int, d_frees: int, nf: int, d_status: int, d_sizes: int, na: int, d_out: int,
                    stream: int = 0) -> None:
    """hba_step with scratch from the library's static device array (no allocation)."""
    check("hba_step_static", _lib().hba_step_static(h, d_frees, nf, d_status, d_sizes, na, d_out, stream))


def hba_reset(h: int, stream: int = 0) -> None:
    check("hba_reset", _lib().hba_reset(h, stream))


def hba_stats(h: int) -> dict:
    s = Stats()
    check("hba_stats", _lib().hba_stats(h, ctypes.byref(s)))
    return s.as_dict()


def hba_export_state(h: int, arena: int = 0) -> np.ndarray:
    n = ctypes.c_size_t()
    check("hba_export_state", _lib().hba_export_state(h, arena, None, 0, ctypes.byref(n)))
    buf = np.empty(n.value, dtype=np.uint64)
    check("hba_export_state", _lib().hba_export_state(h, arena, buf.ctypes.data, n.value, ctypes.byref(n)))
    return buf


def hba_multi_create(arena_bytes, min_block: int, policy: int = HBA_POLICY_SEGFIT, max_total_frees: int = 1 << 22) -> int:
    a = np.ascontiguousarray(arena_bytes, dtype=np.uint64)
    h = ctypes.c_void_p()
    check("hba_multi_create", _lib().hba_multi_create(a.size, a.ctypes.data, min_block, policy,
                                                      max_total_frees, ctypes.byref(h)))
    return h.value


def hba_multi_step(h: int, d_free_rowptr: int, d_frees: int, nf_total: int, d_alloc_rowptr: int,
                   d_sizes: int, na_total: int, d_out: int, d_free_status: int, stream: int = 0) -> None:
    check("hba_multi_step", _lib().hba_multi_step(h, d_free_rowptr, d_frees, nf_total, d_alloc_rowptr,
                                                  d_sizes, na_total, d_out, d_free_status, stream))


def hba_multi_create_ex(arena_bytes, min_block: int, policy: int = HBA_POLICY_SEGFIT, max_total_frees: int = 1 << 22,
                        max_total_allocs: int = 0) -> int:
    a = np.ascontiguousarray(arena_bytes, dtype=np.uint64)
    h = ctypes.c_void_p()
    check("hba_multi_create_ex", _lib().hba_multi_create_ex(a.size, a.ctypes.data, min_block, policy, max_total_frees,
                                                            max_total_allocs, ctypes.byref(h)))
    return h.value


def hba_multi_step_host_async(h: int, h_free_rowptr: int, h_frees: int, nf_total: int, h_alloc_rowptr: int,
                              h_sizes: int, na_total: int, h_out: int, h_free_status: int, stream: int = 0) -> None:
    check("hba_multi_step_host_async",
          _lib().hba_multi_step_host_async(h, h_free_rowptr, h_frees, nf_total, h_alloc_rowptr, h_sizes, na_total,
                                           h_out, h_free_status, stream))


def hba_set_shape(h: int, threads: int, ctas: int = 0, smem_bytes: int = 0) -> None:
    check("hba_set_shape", _lib().hba_set_shape(h, threads, ctas, smem_bytes))


HBA_REJECTED = 0xFFFFFFFFFFFFFFFE
HBA_ERR_STATE = 5


def hba_serve_run(h: int, d_arrivals: int, n: int, d_served: int, d_log: int, log_cap: int,
                  queue_depth: int = 0, max_batch: int = 0, bucket_ns: int = 0, time_limit_ns: int = 0,
                  max_ticks: int = 0, stream: int = 0) -> dict:
    """Returns the run's report.  When the run stopped on a full
    free-timing wheel (HBA_ERR_STATE), the HbaError raised carries the
    report as ``.report``."""
    cfg = ServeConfig(queue_depth, max_batch, bucket_ns, time_limit_ns, max_ticks)
    rep = ServeReport()
    code = _lib().hba_serve_run(h, d_arrivals, n, d_served, d_log, log_cap, ctypes.byref(cfg), ctypes.byref(rep),
                                stream)
    if code == HBA_ERR_STATE:
        err = HbaError("hba_serve_run", code)
        err.report = rep.as_dict()
        raise err
    check("hba_serve_run", code)
    return rep.as_dict()


def serve(alloc: "Allocator", arrivals: np.ndarray, log_cap: int | None = None, **cfg):
    """Run the serving loop on ``arrivals`` (uint64[n, 3]: arrival ns, bytes,
    hold ns).  Returns ``(served uint64[n, 3], log uint32[], report)``.  If
    the run stopped on a full free-timing wheel, the HbaError raised carries
    ``.report``, ``.served`` and ``.log`` of the run."""
    torch = _torch()
    arr = np.ascontiguousarray(arrivals, dtype=np.uint64).reshape(-1, 3)
    n = arr.shape[0]
    dev = torch.device("cuda", torch.cuda.current_device())
    d_arr = torch.from_numpy(arr.view(np.int64)).to(dev)
    d_served = torch.empty((max(n, 1), 3), dtype=torch.int64, device=dev)
    cap = log_cap if log_cap is not None else 4 * n + 1024
    d_log = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    try:
        rep = hba_serve_run(alloc.h, _ptr(d_arr), n, _ptr(d_served), _ptr(d_log), cap, **cfg,
                            stream=_stream_ptr(None))
    except HbaError as e:
        if hasattr(e, "report"):
            e.served = d_served[:n].cpu().numpy().view(np.uint64)
            e.log = d_log[:min(cap, e.report["log_words"])].cpu().numpy().view(np.uint32)
        raise
    served = d_served[:n].cpu().numpy().view(np.uint64)
    log = d_log[:min(cap, rep["log_words"])].cpu().numpy().view(np.uint32)
    return served, log, rep


def log_batches(log: np.ndarray):
    """Split a serving tick log into (free ids, alloc ids) per tick."""
    out, i = [], 0
    while i + 2 <= log.size:
        nf, na = int(log[i]), int(log[i + 1])
        out.append((log[i + 2:i + 2 + nf], log[i + 2 + nf:i + 2 + nf + na]))
        i += 2 + nf + na
    return out


def hba_version() -> str:
    return _lib().hba_version().decode()


def hba_launch_count(h: int) -> int:
    """Kernels the handle has launched so far."""
    c = ctypes.c_uint64(0)
    check("hba_launch_count", _lib().hba_launch_count(h, ctypes.byref(c)))
    return c.value


# ---- torch convenience wrappers ----------------------------------------------

def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr()) if t is not None and t.numel() else 0


class Allocator:
    """One arena.  Inputs/outputs are uint64 (int64-typed) CUDA tensors."""

    def __init__(self, arena_bytes: int, min_block: int, max_batch: int = 65536, threads: int | None = None,
                 smem_bytes: int = 0, ctas: int = 0, policy: str = "segfit"):
        """``ctas``: size of the batch's thread-block cluster (0 or 1: a
        separate gathering grid, then the engine; 2..8: the engine CTA plus
        gathering CTAs; see hba_set_shape).  ``policy``: "segfit" (§5.1),
        "tlsf" (§5.2), the sequential fits "first", "next", "best" (§4),
        or the bitmask pool "bitmask" (§3.2)."""
        self.policy = policy
        self.h = hba_create(arena_bytes, min_block, POLICIES[policy], max_batch)
        self.arena_bytes = arena_bytes - arena_bytes % min_block
        self.min_block = min_block
        self.max_batch = max_batch
        if threads is not None or smem_bytes or ctas:
            hba_set_shape(self.h, threads or 1024, ctas, smem_bytes)

    def close(self):
        if self.h:
            hba_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, frees=None, sizes=None, out=None, status=None, stream=None):
        """Frees (index order), then allocations (index order), one launch."""
        torch = _torch()
        nf = 0 if frees is None else frees.numel()
        na = 0 if sizes is None else sizes.numel()
        if na and out is None:
            out = torch.empty(na, dtype=torch.int64, device=sizes.device)
        hba_step(self.h, _ptr(frees), nf, _ptr(status), _ptr(sizes), na, _ptr(out), _stream_ptr(stream))
        return out

    def alloc_batch(self, sizes, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(sizes.numel(), dtype=torch.int64, device=sizes.device)
        hba_alloc_batch(self.h, _ptr(sizes), sizes.numel(), _ptr(out), _stream_ptr(stream))
        return out

    def free_batch(self, offsets, status=None, stream=None):
        hba_free_batch_ex(self.h, _ptr(offsets), offsets.numel(), _ptr(status), _stream_ptr(stream))

    def reset(self, stream=None):
        hba_reset(self.h, _stream_ptr(stream))

    def stats(self) -> dict:
        return hba_stats(self.h)

    def launches(self) -> int:
        return hba_launch_count(self.h)

    def export_state(self) -> np.ndarray:
        return hba_export_state(self.h, 0)


class MultiAllocator:
    """Many independent arenas; one launch applies one batch to all of them."""

    def __init__(self, arena_bytes, min_block: int, max_total_frees: int = 1 << 22, policy: str = "segfit",
                 max_total_allocs: int = 0):
        """``max_total_allocs`` > 0 gives the handle staging for
        hba_multi_step_host_async (batches from host buffers)."""
        self.policy = policy
        self.h = (hba_multi_create_ex(arena_bytes, min_block, POLICIES[policy], max_total_frees, max_total_allocs)
                  if max_total_allocs else hba_multi_create(arena_bytes, min_block, POLICIES[policy], max_total_frees))
        self.n = len(arena_bytes)

    def close(self):
        if self.h:
            hba_destroy(self.h)
            self.h = 0

    def set_shape(self, threads: int, ctas: int = 0, smem_bytes: int = 0):
        hba_set_shape(self.h, threads, ctas, smem_bytes)

    def step(self, free_rowptr, frees, alloc_rowptr, sizes, out, status=None, stream=None):
        hba_multi_step(self.h, _ptr(free_rowptr), _ptr(frees), frees.numel(), _ptr(alloc_rowptr),
                       _ptr(sizes), sizes.numel(), _ptr(out), _ptr(status), _stream_ptr(stream))

    def stats(self) -> dict:
        return hba_stats(self.h)

    def export_state(self, arena: int) -> np.ndarray:
        return hba_export_state(self.h, arena)


__all__ = ([n for n in dir() if n.startswith(("hba_", "HBA_"))]
           + ["Allocator", "MultiAllocator", "HbaError", "serve", "log_batches"])
