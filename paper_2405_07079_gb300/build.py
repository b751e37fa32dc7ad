"""Build the CUDA library ``_build/libhba.so`` for sm_103a with nvcc.

The library is compiled in-tree (never installed) from ``csrc/hba_capi.cu``
and the kernel headers it includes (``csrc/*.cuh``); the public header is
``include/hba.h`` at the repository root.  ``_build/libcuda_replay.so`` (host code only, from
``csrc/cuda_replay.cu``) replays traces through the CUDA runtime's own
allocators for the benchmark's comparison; it is compiled alongside.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libhba.so")
SOURCES = [os.path.join(CSRC, "hba_capi.cu")]
DEPS = SOURCES + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "hba.h")]
REPLAY_LIB = os.path.join(BUILD, "libcuda_replay.so")
REPLAY_SOURCES = [os.path.join(CSRC, "cuda_replay.cu")]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile both libraries (in parallel) when stale; returns the path of libhba.so."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for target, sources, deps in ((LIB, SOURCES, DEPS), (REPLAY_LIB, REPLAY_SOURCES, REPLAY_SOURCES)):
        if force or stale(target, deps):
            tmp = target + f".tmp{os.getpid()}"
            cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-o", tmp, *sources]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            jobs.append((subprocess.Popen(cmd), tmp, target, cmd))
    for proc, tmp, target, cmd in jobs:
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, cmd)
        os.replace(tmp, target)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
