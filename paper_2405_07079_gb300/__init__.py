"""Header-free batched allocator for GB300 (sm_103a).

The segregated-fit allocator of Bell, Kumar and Gill, "Host-Based Allocators
for Device Memory" (arXiv 2405.07079, §5.1), with all metadata out of band
and batches of malloc/free requests applied on the GPU.  The C ABI is in
``include/hba.h``; ``hba`` is its Python binding, re-exported here whole:
one function per C entry point, the constants, and the torch wrappers.
"""
from . import hba as _hba
from .hba import *  # noqa: F401,F403

__all__ = list(_hba.__all__)
