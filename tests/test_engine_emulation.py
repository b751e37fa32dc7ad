"""The batch engine's logic, compiled for the host (HBA_EMULATE), against the
oracle.  The kernel body runs phase by phase as loops over thread indices;
small CTA widths force many chunk boundaries.  This checks the parallel
formulation (run detection, list surgery, carve chunks) without a GPU; the
GPU tests check the same source on the device."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

from _helpers import oracle_trace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_07079_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "emu", "hba_emu.cpp")
HDR = os.path.join(CSRC, "hba_engine.cuh")
TLSF_HDR = os.path.join(CSRC, "hba_tlsf.cuh")
OUT = os.path.join(ROOT, "tests", "emu", "_build", "libhba_emu_test.so")


@pytest.fixture(scope="module")
def emu():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(map(os.path.getmtime, (SRC, HDR, TLSF_HDR))):
        tmp = OUT + f".{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", tmp, SRC])
        os.replace(tmp, OUT)
    lib = ctypes.CDLL(OUT)
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    lib.emu_create.restype = vp
    lib.emu_create.argtypes = [u64, u64, ctypes.c_int]
    lib.emu_destroy.argtypes = [vp]
    lib.emu_step.argtypes = [vp, vp, u32, vp, vp, u32, vp]
    lib.emu_export.restype = ctypes.c_size_t
    lib.emu_export.argtypes = [vp, vp, ctypes.c_size_t]
    lib.emu_stats.argtypes = [vp, vp]
    lib.emu_set_dyn.argtypes = [vp, u32]
    lib.emu_set_staged.argtypes = [vp, ctypes.c_int]
    lib.emu_set_self.argtypes = [vp, ctypes.c_int]
    lib.emu_set_tlsf.argtypes = [vp]
    lib.emu_export_tlsf.restype = ctypes.c_size_t
    lib.emu_export_tlsf.argtypes = [vp, vp, ctypes.c_size_t]
    lib.emu_tlsf_create.restype = vp
    lib.emu_tlsf_create.argtypes = [u64, u64]
    lib.emu_tlsf_destroy.argtypes = [vp]
    lib.emu_tlsf_step.argtypes = [vp, vp, u32, vp, vp, u32, vp]
    lib.emu_tlsf_export.restype = ctypes.c_size_t
    lib.emu_tlsf_export.argtypes = [vp, vp, ctypes.c_size_t]
    lib.emu_tlsf_stats.argtypes = [vp, vp]
    return lib


class Emu:
    def __init__(self, lib, A, mb, nt, dyn_words=None, staged=False, self_gather=False, tlsf=False):
        self.lib, self.h = lib, lib.emu_create(A, mb, nt)
        assert self.h
        self.tlsf = tlsf
        if tlsf:
            lib.emu_set_tlsf(self.h)
        if dyn_words is not None:
            lib.emu_set_dyn(self.h, dyn_words)
        lib.emu_set_staged(self.h, int(staged))
        lib.emu_set_self(self.h, int(self_gather))

    def batch(self, f, s):
        f = np.ascontiguousarray(f, np.uint64)
        s = np.ascontiguousarray(s, np.uint64)
        out = np.empty(s.size, np.uint64)
        st = np.empty(f.size, np.uint8)
        p = lambda a: a.ctypes.data if a.size else None
        assert self.lib.emu_step(self.h, p(f), f.size, p(st), p(s), s.size, p(out)) == 0
        return out, st

    def export_state(self):
        fn = self.lib.emu_export_tlsf if self.tlsf else self.lib.emu_export
        n = fn(self.h, None, 0)
        b = np.empty(n, np.uint64)
        fn(self.h, b.ctypes.data, n)
        return b

    def stats(self):
        b = np.zeros(9, np.uint64)
        self.lib.emu_stats(self.h, b.ctypes.data)
        return [int(x) for x in b]

    def close(self):
        self.lib.emu_destroy(self.h)


def _check(emu, wl, nt, every=1, dyn_words=None, staged=False, self_gather=False):
    trace, o = oracle_trace(wl)
    e = Emu(emu, wl.arena, wl.min_block, nt, dyn_words, staged, self_gather)
    import oracle as _o
    ref = _o.Oracle(wl.arena, wl.min_block)
    try:
        for b, (f, s, out, st) in enumerate(trace):
            go, gs = e.batch(f, s)
            ref.batch(f, s)
            assert np.array_equal(go, out), f"batch {b} allocs"
            assert np.array_equal(gs, st), f"batch {b} frees"
            if b % every == 0:
                assert np.array_equal(e.export_state(), ref.export_state()), f"batch {b} state"
        assert np.array_equal(e.export_state(), o.export_state())
        assert e.stats() == list(o.stats().values())
    finally:
        e.close()


@pytest.mark.parametrize("nt", [4, 32, 256, 1024])
def test_tiny(emu, nt):
    from paper_2405_07079_gb300 import workloads as W
    _check(emu, W.tiny(n_ops=4000 if nt == 4 else 10_000), nt)


@pytest.mark.parametrize("nt", [4, 32, 256])
def test_dense_random(emu, nt):
    from paper_2405_07079_gb300 import workloads as W
    wl = W.Workload("dense", 1 << 20, 256, lambda: W.TinyRandom(n_ops=4000, batch=400, p_free=0.5))
    _check(emu, wl, nt)


@pytest.mark.parametrize("dyn_words", [0, 4096, 1 << 20])
def test_scratch_placements(emu, dyn_words):
    """Free-phase scratch all in global memory, pointer jumping only in shared
    memory, and everything in shared memory."""
    from paper_2405_07079_gb300 import workloads as W
    wl = W.Workload("life", 1 << 28, 512, lambda: W.Lifetimes(n_ops=200_000, batch=4096, mean_life=60))
    _check(emu, wl, 256, every=3, dyn_words=dyn_words)


@pytest.mark.parametrize("nt", [32, 256])
def test_lifetimes(emu, nt):
    from paper_2405_07079_gb300 import workloads as W
    wl = W.Workload("life", 1 << 30, 512, lambda: W.Lifetimes(n_ops=300_000, batch=8192, mean_life=100))
    _check(emu, wl, nt, every=4)


@pytest.mark.parametrize("nt", [256, 1024])
def test_staged_by_cluster(emu, nt):
    """The gathered records written straight into the free phase's shared
    memory (what the gathering CTAs of a cluster do), with the table and the
    per-free arrays after them."""
    from paper_2405_07079_gb300 import workloads as W
    wl = W.Workload("life", 1 << 28, 512, lambda: W.Lifetimes(n_ops=200_000, batch=4096, mean_life=60))
    _check(emu, wl, nt, every=3, dyn_words=1 << 20, staged=True)
    _check(emu, W.tiny(n_ops=6000), nt, dyn_words=1 << 20, staged=True)


@pytest.mark.parametrize("nt,dyn_words", [(4, None), (256, 1 << 20), (256, 0), (1024, 1 << 20)])
def test_self_gather(emu, nt, dyn_words):
    """The engine gathers its frees' records itself (no gathering grid), into
    the shared-memory layout when it fits, else into the global buffer."""
    from paper_2405_07079_gb300 import workloads as W
    _check(emu, W.tiny(n_ops=6000), nt, dyn_words=dyn_words, self_gather=True)
    wl = W.Workload("life", 1 << 28, 512, lambda: W.Lifetimes(n_ops=100_000, batch=2048, mean_life=60))
    _check(emu, wl, nt, every=5, dyn_words=dyn_words, self_gather=True)


@pytest.mark.parametrize("nt", [32, 1024])
def test_frag(emu, nt):
    from paper_2405_07079_gb300 import workloads as W
    _check(emu, W.frag(n_fill=30_000, n_big=3000, batch=2048, arena=1 << 27), nt, every=3)


def test_many_small_arenas_random(emu):
    """Tiny arenas with every op kind, including invalid and duplicate frees."""
    import oracle
    rng = np.random.default_rng(1)
    for trial in range(150):
        mb = int(rng.choice([8, 16, 256]))
        A = mb * int(rng.integers(1, 200))
        nt = int(rng.choice([4, 32]))
        o, e = oracle.Oracle(A, mb), Emu(emu, A, mb, nt)
        held = []
        for _ in range(25):
            fr = [held[int(rng.integers(0, len(held)))] if held and rng.random() < 0.8
                  else int(rng.integers(0, A + mb)) for _ in range(int(rng.integers(0, 12)))]
            sz = [int(x) for x in rng.integers(0, A + 2 * mb, int(rng.integers(0, 12)))]
            f, s = np.array(fr, np.uint64), np.array(sz, np.uint64)
            oo, os_ = o.batch(f, s)
            eo, es = e.batch(f, s)
            assert np.array_equal(oo, eo) and np.array_equal(os_, es), trial
            assert np.array_equal(o.export_state(), e.export_state()), trial
            held = [a for a in held if a not in set(fr)] + [int(x) for x in oo if x != 0xFFFFFFFFFFFFFFFF]
        e.close()


def _check_tlsf(emu, wl, every=1):
    """The TLSF per-op functions of the GPU kernel, applied one request at a
    time on the host, against the TLSF oracle: every result, every status,
    the canonical state (lists and both bitmap levels) and the counters."""
    import oracle as _o

    ref = _o.Oracle(wl.arena, wl.min_block, "tlsf")
    h = emu.emu_tlsf_create(wl.arena, wl.min_block)
    assert h
    p = lambda a: a.ctypes.data if a.size else None

    def export():
        n = emu.emu_tlsf_export(h, None, 0)
        b = np.empty(n, np.uint64)
        emu.emu_tlsf_export(h, b.ctypes.data, n)
        return b

    try:
        cl = wl.make()
        b = 0
        while (req := cl.next_batch()) is not None:
            f = np.ascontiguousarray(req[0], np.uint64)
            s = np.ascontiguousarray(req[1], np.uint64)
            out = np.empty(s.size, np.uint64)
            st = np.empty(f.size, np.uint8)
            emu.emu_tlsf_step(h, p(f), f.size, p(st), p(s), s.size, p(out))
            ro, rs = ref.batch(f, s)
            cl.feed(ro)
            assert np.array_equal(out, ro), f"batch {b} allocs"
            assert np.array_equal(st, rs), f"batch {b} frees"
            if b % every == 0:
                assert np.array_equal(export(), ref.export_state()), f"batch {b} state"
            b += 1
        assert np.array_equal(export(), ref.export_state())
        got = np.zeros(9, np.uint64)
        emu.emu_tlsf_stats(h, got.ctypes.data)
        assert [int(x) for x in got] == list(ref.stats().values())
    finally:
        emu.emu_tlsf_destroy(h)


def test_tlsf_ops_on_workloads(emu):
    from paper_2405_07079_gb300 import workloads as W

    _check_tlsf(emu, W.tiny(n_ops=6000))
    _check_tlsf(emu, W.usage(n_ops=3000, batch=8), every=10)
    _check_tlsf(emu, W.Workload("life", 1 << 28, 512, lambda: W.Lifetimes(n_ops=60_000, batch=2048, mean_life=100)),
                every=4)
    _check_tlsf(emu, W.frag(n_fill=20_000, n_big=2000, batch=2048, arena=1 << 27), every=5)


def test_tlsf_ops_on_small_random_arenas(emu):
    """Tiny arenas of 8-byte to 256-byte granules (list classes below the
    second-level split, exact lists), every op kind including invalid and
    duplicate frees."""
    from paper_2405_07079_gb300 import workloads as W

    for mb, G in ((8, 37), (16, 200), (256, 1000), (8, 3)):
        _check_tlsf(emu, W.Workload("t", mb * G, mb, lambda: W.TinyRandom(n_ops=3000, batch=7, p_free=0.45,
                                                                        lo=1, hi=mb * G // 3 + 1)))


def _check_engine_tlsf(emu, wl, nt, every=1, dyn_words=None, self_gather=False):
    """Two-level segregated fit through the parallel batch engine (the
    engine's second class layout) against the TLSF oracle: every result,
    every free status, the canonical state (lists and both bitmap levels)
    and the counters."""
    trace, o = oracle_trace(wl, policy="tlsf")
    e = Emu(emu, wl.arena, wl.min_block, nt, dyn_words, False, self_gather, tlsf=True)
    import oracle as _o
    ref = _o.Oracle(wl.arena, wl.min_block, "tlsf")
    try:
        for b, (f, s, out, st) in enumerate(trace):
            go, gs = e.batch(f, s)
            ref.batch(f, s)
            assert np.array_equal(go, out), f"batch {b} allocs"
            assert np.array_equal(gs, st), f"batch {b} frees"
            if b % every == 0:
                assert np.array_equal(e.export_state(), ref.export_state()), f"batch {b} state"
        assert np.array_equal(e.export_state(), o.export_state())
        assert e.stats() == list(o.stats().values())
    finally:
        e.close()


@pytest.mark.parametrize("nt", [4, 32, 256, 1024])
def test_engine_tlsf_tiny(emu, nt):
    from paper_2405_07079_gb300 import workloads as W

    _check_engine_tlsf(emu, W.tiny(n_ops=4000 if nt == 4 else 8000), nt, every=3)


@pytest.mark.parametrize("nt,dyn_words", [(32, None), (256, 0), (256, 1 << 20), (1024, 1 << 20)])
def test_engine_tlsf_lifetimes(emu, nt, dyn_words):
    """Many runs a batch (the push by same-list predecessors), free phases in
    shared memory and in global scratch."""
    from paper_2405_07079_gb300 import workloads as W

    wl = W.Workload("life", 1 << 26, 512, lambda: W.Lifetimes(n_ops=60_000, batch=4096, mean_life=300,
                                                            scale=1 / 64, min_size=512))
    _check_engine_tlsf(emu, wl, nt, every=4, dyn_words=dyn_words)


def test_engine_tlsf_usage_and_small_arenas(emu):
    from paper_2405_07079_gb300 import workloads as W

    _check_engine_tlsf(emu, W.usage(n_ops=1500, batch=16), 256, every=5)
    rng = np.random.default_rng(12)
    for _ in range(40):
        mb = int(rng.choice([8, 16, 256]))
        A = mb * int(rng.integers(1, 300))
        wl = W.Workload("small", A, mb, lambda A=A, mb=mb: W.TinyRandom(n_ops=400, batch=int(rng.integers(1, 40)),
                                                                       lo=1, hi=A))
        _check_engine_tlsf(emu, wl, int(rng.choice([4, 32])))
