"""Header-free batched allocator for GB300 (sm_103a).

The segregated-fit allocator of Bell, Kumar and Gill, "Host-Based Allocators
for Device Memory" (arXiv 2405.07079, §5.1), with all metadata out of band
and batches of malloc/free requests applied on the GPU.  The C ABI is in
``include/hba.h``; ``hba`` is its Python binding.
"""
from .hba import (HBA_FAIL, HBA_POLICY_SEGFIT, HBA_POLICY_TLSF, Allocator, HbaError, MultiAllocator, hba_alloc_batch, hba_create,
                  hba_destroy, hba_export_state, hba_free_batch, hba_free_batch_ex, hba_multi_create,
                  hba_set_shape, hba_multi_step, hba_reset, hba_stats, hba_step, hba_step_host,
                  hba_step_host_async, hba_step_static, hba_version, hba_launch_count, HBA_STATIC_MAX_FREES,
                  hba_serve_run, HBA_REJECTED, serve, log_batches)

__all__ = ["HBA_FAIL", "HBA_POLICY_SEGFIT", "HBA_POLICY_TLSF", "Allocator", "HbaError", "MultiAllocator", "hba_alloc_batch", "hba_create",
           "hba_destroy", "hba_export_state", "hba_free_batch", "hba_free_batch_ex", "hba_multi_create",
           "hba_set_shape", "hba_multi_step", "hba_reset", "hba_stats", "hba_step", "hba_step_host",
           "hba_step_host_async", "hba_step_static", "hba_version", "hba_launch_count", "HBA_STATIC_MAX_FREES", "hba_serve_run", "HBA_REJECTED", "serve",
           "log_batches"]
