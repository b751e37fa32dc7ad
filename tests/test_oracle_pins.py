"""Pins of the CPU oracle to things other than itself (no GPU needed).

* hand-derived worked examples (tests/golden/worked_examples.json);
* closed forms (carving prefix sums, the fragmentation fill, a full arena of
  4 KiB holes, release-all returns one block, exact powers of two);
* invariants of every intermediate state;
* an independent brute-force restatement (oracle/interval_ref.py), exhaustive
  on tiny arenas and on random traces;
* mutation checks: plausible mistakes planted in the brute-force restatement
  (FIFO lists, 1-based class, lenient class, floor class) are caught by the
  worked examples.
"""
from __future__ import annotations

import itertools
import json
import os

import numpy as np
import pytest

from _helpers import check_invariants

import oracle
from oracle.interval_ref import IntervalAllocator, _ceil_log2, _floor_log2

FAIL = 0xFFFFFFFFFFFFFFFF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _canonical(arena, min_block, blocks, lists, bitmask):
    w = [arena, min_block, len(blocks)]
    for off, size, free in blocks:
        w += [off, size | (int(free) << 63)]
    for k in range(64):
        lst = lists.get(str(k), [])
        w += [len(lst)] + list(lst)
    return w + [bitmask]


def load_golden():
    with open(GOLDEN) as f:
        doc = json.load(f)
    cases = []
    for c in doc["cases"]:
        fin = c.get("final")
        if fin is not None:
            blocks = fin["blocks"]
            if isinstance(blocks, str):  # "pages:<size>:<count>:free=<offset>"
                _, sz, cnt, fr = blocks.split(":")
                sz, cnt, fr = int(sz), int(cnt), int(fr.split("=")[1])
                blocks = [[i * sz, sz, i * sz == fr] for i in range(cnt)]
            words = _canonical(c["arena"], c["min_block"], blocks, fin["lists"], fin["bitmask"])
        else:
            words = None
        cases.append({"name": c["name"], "arena": c["arena"], "min_block": c["min_block"],
                      "batches": c["batches"], "final": words})
    return cases


@pytest.mark.parametrize("impl", [oracle.Oracle, IntervalAllocator])
@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"].split()[0])
def test_worked_example(impl, case):
    a = impl(case["arena"], case["min_block"])
    for frees, sizes, expect in case["batches"]:
        out, st = a.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        assert [int(x) for x in out] == expect
        assert all(int(s) == 0 for s in st), "every free in the worked examples is valid"
    assert [int(x) for x in a.export_state()] == case["final"]


# ---- mutation checks: the worked examples catch plausible mistakes ---------

class _Fifo(IntervalAllocator):
    """Lists used as queues (pop the OLDEST push)."""

    def malloc(self, size):
        for v in self.iv:
            v[3] = -v[3] if v[2] else v[3]
        try:
            return super().malloc(size)
        finally:
            for v in self.iv:
                v[3] = -v[3] if v[2] and v[3] < 0 else v[3]


class _ClassShift(IntervalAllocator):
    """Class off by `shift` (1-based ffs reading: +1; lenient: -1)."""
    shift = 1

    def malloc(self, size):
        if size == 0 or size > self.arena:
            return FAIL
        s = -(-size // self.min_block) * self.min_block
        c = max(0, _ceil_log2(s) + self.shift)
        cands = [(_floor_log2(v[1]), -v[3], k) for k, v in enumerate(self.iv)
                 if v[2] and _floor_log2(v[1]) >= c and v[1] >= s]
        if not cands:
            return FAIL
        k = min(cands)[2]
        st, sz = self.iv[k][0], self.iv[k][1]
        self.iv[k] = [st, s, False, 0]
        if sz > s:
            self.iv.insert(k + 1, [st + s, sz - s, True, self._tick()])
        return st


class _Lenient(_ClassShift):
    shift = -1


class _FloorClass(_ClassShift):
    """Class floor(log2 s') instead of ceil (may pick a block that is too small
    in class but large enough in bytes)."""

    def malloc(self, size):
        if size == 0 or size > self.arena:
            return FAIL
        s = -(-size // self.min_block) * self.min_block
        self.shift = _floor_log2(s) - _ceil_log2(s)
        return super().malloc(size)


class _NoMerge(IntervalAllocator):
    """Frees never coalesce."""

    def free(self, addr):
        k = next((i for i, v in enumerate(self.iv) if v[0] == addr), None)
        if k is None or self.iv[k][2]:
            return 1
        self.iv[k][2] = True
        self.iv[k][3] = self._tick()
        return 0


@pytest.mark.parametrize("mutant", [_Fifo, _ClassShift, _Lenient, _FloorClass, _NoMerge])
def test_worked_examples_catch_mutants(mutant):
    caught = False
    for case in load_golden():
        a = mutant(case["arena"], case["min_block"])
        ok = True
        for frees, sizes, expect in case["batches"]:
            out, _ = a.batch(frees, sizes)
            ok &= [int(x) for x in out] == expect
        ok &= [int(x) for x in a.export_state()] == case["final"]
        caught |= not ok
    assert caught, f"{mutant.__name__} passes every worked example"


# ---- closed forms -------------------------------------------------------------

def test_nearly_four_times_bound():
    """With the request's own class non-empty, the chosen block is < 4x the
    rounded request (§5.1, text after Algorithm 4): class c = ceil(log2 s')
    holds blocks below 2^(c+1) < 4 s'."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        mb = 256
        o = oracle.Oracle(1 << 24, mb)
        held = [o.malloc(int(x)) for x in rng.integers(1, 1 << 16, 60)]
        for a in held[::2]:
            if a != FAIL:
                o.free(a)
        st = oracle.decode_state(o.export_state())
        size_of = {off: sz for off, sz, fr in st["blocks"] if fr}
        for s in rng.integers(1, 1 << 16, 20):
            sp = -(-int(s) // mb) * mb
            c = _ceil_log2(sp)
            if st["bins"][c]:
                head = st["bins"][c][0]
                assert o.malloc(int(s)) == head and size_of[head] < 4 * sp
                break


def test_carving_prefix_sums():
    """From a fresh arena, allocations carve the front: offset_i = sum of the
    earlier rounded sizes while the request's class fits the remainder."""
    rng = np.random.default_rng(5)
    for trial in range(50):
        A, mb = 1 << 22, 1 << int(rng.integers(3, 10))
        o = oracle.Oracle(A, mb)
        used = 0
        for s in rng.integers(1, 1 << 14, 100):
            sp = -(-int(s) // mb) * mb
            rem = A - used
            expect = used if rem > 0 and (1 << _ceil_log2(sp)) <= rem else FAIL
            assert o.malloc(int(s)) == expect
            if expect != FAIL:
                used += sp
            # the carved prefix is the extent; the rest is one free block
            assert o.space() == {"extent": used, "largest_free": A - used}


def test_frag_fill_and_full_arena_closed_forms():
    """Fill with 4 KiB blocks -> offsets 4096 i.  With an arena of exactly
    n x 4 KiB, after freeing every other block all holes are 4 KiB (class 12)
    and any request of class >= 13 fails."""
    n = 4096
    o = oracle.Oracle(n * 4096, 256)
    out, _ = o.batch(np.zeros(0, np.uint64), np.full(n, 4096, np.uint64))
    assert np.array_equal(out, np.arange(n, dtype=np.uint64) * 4096)
    assert o.space() == {"extent": n * 4096, "largest_free": 0}
    _, st = o.batch(out[0::2], np.zeros(0, np.uint64))
    assert not st.any()
    # the last block (odd index) stays in use: the extent does not shrink
    assert o.space() == {"extent": n * 4096, "largest_free": 4096}
    out2, _ = o.batch(np.zeros(0, np.uint64), np.array([4097, 8192, 1 << 20], np.uint64))
    assert (out2 == FAIL).all()
    s = oracle.decode_state(o.export_state())
    assert s["bitmask"] == 1 << 12 and len(s["bins"][12]) == n // 2


def test_space_of_the_first_worked_example():
    """W1 (A = 4096, min block 256) batch by batch: extent = end of the
    highest in-use block, largest free block from the free blocks left."""
    u = lambda *v: np.array(v, dtype=np.uint64)
    o = oracle.Oracle(4096, 256)
    assert o.space() == {"extent": 0, "largest_free": 4096}
    o.batch(u(), u(1000, 256, 3000))                  # [0,1024) [1024,1280) used
    assert o.space() == {"extent": 1280, "largest_free": 4096 - 1280}
    o.batch(u(0), u(2048))                            # [1280,3328) used, [0,1024) free
    assert o.space() == {"extent": 3328, "largest_free": 1024}
    o.batch(u(1024, 1280), u(512))                    # everything merged, then [0,512)
    assert o.space() == {"extent": 512, "largest_free": 3584}


def test_release_all_returns_one_block():
    rng = np.random.default_rng(9)
    for trial in range(20):
        o = oracle.Oracle(1 << 22, 512)
        held = []
        for _ in range(30):
            out, _ = o.batch(np.zeros(0, np.uint64), rng.integers(1, 1 << 17, 40).astype(np.uint64))
            held += [int(x) for x in out if x != FAIL]
            if held and rng.random() < 0.5:
                k = int(rng.integers(0, len(held)))
                o.free(held.pop(k))
        order = rng.permutation(len(held))
        _, st = o.batch(np.array(held, np.uint64)[order], np.zeros(0, np.uint64))
        assert not st.any()
        s = oracle.decode_state(o.export_state())
        assert s["blocks"] == [(0, 1 << 22, True)] and s["bins"][22] == [0]
        assert o.space() == {"extent": 0, "largest_free": 1 << 22}


def test_exact_powers_of_two_fit_from_own_class():
    o = oracle.Oracle(1 << 20, 256)
    for k in range(8, 20):
        o2 = oracle.Oracle(1 << 20, 256)
        o2.malloc(1 << 19)  # leaves [2^19, 2^20) in class 19
        if k <= 19:
            assert o2.malloc(1 << k) == 1 << 19
    assert o.malloc(1 << 20) == 0 and o.malloc(256) == FAIL


# ---- invariants and brute force -------------------------------------------

def _random_batches(rng, A, mb, nb, max_ops, sizes_hi):
    held = []
    for _ in range(nb):
        nf = int(rng.integers(0, max_ops + 1))
        frees = []
        for _ in range(nf):
            r = rng.random()
            if held and r < 0.7:
                frees.append(held[int(rng.integers(0, len(held)))])
            elif r < 0.85:
                frees.append(int(rng.integers(0, A // mb + 2)) * mb)   # maybe a non-start
            else:
                frees.append(int(rng.integers(0, A + 64)))              # maybe misaligned
        sizes = [int(x) for x in rng.integers(0, sizes_hi, int(rng.integers(0, max_ops + 1)))]
        yield frees, sizes, held


@pytest.mark.parametrize("seed", range(40))
def test_oracle_equals_interval_allocator_random(seed):
    rng = np.random.default_rng(seed)
    mb = [8, 16, 64][seed % 3]
    A = mb * int(rng.integers(1, 40))
    o, r = oracle.Oracle(A, mb), IntervalAllocator(A, mb)
    for frees, sizes, held in _random_batches(rng, A, mb, 40, 6, A + mb):
        oo, os_ = o.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        ro, rs = r.batch(frees, sizes)
        assert [int(x) for x in oo] == ro and [int(x) for x in os_] == rs
        assert [int(x) for x in o.export_state()] == r.export_state()
        check_invariants(o.export_state())
        held[:] = [a for a in held if a not in set(frees)] + [int(x) for x in oo if x != FAIL]


def test_oracle_equals_interval_allocator_exhaustive():
    """Every sequence of 4 single-op batches over a small alphabet on a
    16-granule arena, after each of three different prefixes."""
    A, mb = 256, 16
    alphabet = [("a", 1), ("a", 16), ("a", 17), ("a", 48), ("a", 100), ("a", 256),
                ("f", 0), ("f", 16), ("f", 32), ("f", 64), ("f", 128), ("f", 8)]
    prefixes = [[], [("a", 32), ("a", 16), ("a", 64), ("f", 32)], [("a", 16)] * 8 + [("f", 16), ("f", 64)]]
    n = 0
    for pre in prefixes:
        for seq in itertools.product(alphabet, repeat=4):
            o, r = oracle.Oracle(A, mb), IntervalAllocator(A, mb)
            for op, v in list(pre) + list(seq):
                if op == "a":
                    assert o.malloc(v) == r.malloc(v)
                else:
                    assert o.free(v) == r.free(v)
            assert [int(x) for x in o.export_state()] == r.export_state()
            n += 1
    assert n == 3 * len(alphabet) ** 4


def test_invariants_on_workload_traces():
    from paper_2405_07079_gb300 import workloads as W

    for wl in (W.tiny(n_ops=3000),
               W.Workload("l", 1 << 28, 512, lambda: W.Lifetimes(n_ops=60_000, batch=2048, mean_life=200)),
               W.frag(n_fill=8000, n_big=800, batch=1024, arena=64 << 20),
               W.Workload("u", 1 << 28, 4096, lambda: W.RandomSlots(n_ops=3000, slots=48, hi=4 << 20, batch=8))):
        o = oracle.Oracle(wl.arena, wl.min_block)
        cl = wl.make()
        while (b := cl.next_batch()) is not None:
            out, st = o.batch(*b)
            cl.feed(out)
            check_invariants(o.export_state())
            stt = o.stats()
            s = oracle.decode_state(o.export_state())
            assert stt["used_bytes"] == sum(sz for _, sz, fr in s["blocks"] if not fr)
            assert stt["blocks"] == len(s["blocks"])
            # the space report against a walk of the blocks in address order
            sp = o.space()
            assert sp["largest_free"] == max([sz for _, sz, fr in s["blocks"] if fr], default=0)
            assert sp["extent"] == max([off + sz for off, sz, fr in s["blocks"] if not fr], default=0)


def test_random_slots_batches_keep_sequential_order():
    """The malloc-large stand-in cut into batches of up to 16 ops gives the
    same results, op for op, and the same final state as one op per batch:
    its batches never put a malloc before a free or touch a slot twice."""
    from paper_2405_07079_gb300 import workloads as W

    runs = []
    for bs in (1, 16):
        o = oracle.Oracle(1 << 30, 4096)
        cl = W.RandomSlots(n_ops=1500, slots=24, batch=bs)
        ops = []
        while (b := cl.next_batch()) is not None:
            out, st = o.batch(*b)
            cl.feed(out)
            ops += [("f", int(x), int(t)) for x, t in zip(b[0], st)] + [("a", int(x), int(y)) for x, y in zip(b[1], out)]
        runs.append((ops, o.export_state().tolist(), o.space()))
    assert runs[0] == runs[1]
    assert len(runs[0][0]) == 1500


# ---- two-level segregated fit (§5.2) ----------------------------------------
TLSF_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tlsf_worked_examples.json")


def load_tlsf_golden():
    with open(TLSF_GOLDEN) as f:
        doc = json.load(f)
    cases = []
    for c in doc["cases"]:
        fin = c["final"]
        w = [c["arena"], c["min_block"], len(fin["blocks"])]
        for off, size, free in fin["blocks"]:
            w += [off, size | (int(free) << 63)]
        for k in range(64 * 16):
            lst = fin["lists"].get(str(k), [])
            w += [len(lst)] + list(lst)
        w.append(fin["flmask"])
        w += [fin["slmask"].get(str(f), 0) for f in range(64)]
        cases.append({"name": c["name"], "arena": c["arena"], "min_block": c["min_block"],
                      "batches": c["batches"], "final": w})
    return cases


def _tlsf_oracle(A, mb):
    return oracle.Oracle(A, mb, "tlsf")


def _tlsf_interval(A, mb):
    return IntervalAllocator(A, mb, "tlsf")


@pytest.mark.parametrize("make", [_tlsf_oracle, _tlsf_interval])
@pytest.mark.parametrize("case", load_tlsf_golden(), ids=lambda c: c["name"].split()[0])
def test_tlsf_worked_example(make, case):
    a = make(case["arena"], case["min_block"])
    for frees, sizes, expect in case["batches"]:
        out, st = a.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        assert [int(x) for x in out] == expect, case["name"]
        assert not any(int(x) for x in st)
    assert [int(x) for x in a.export_state()] == case["final"], case["name"]


@pytest.mark.parametrize("mutant", ["no_rounding", "eight_lists", "power_of_two_search"])
def test_tlsf_worked_examples_catch_mutants(monkeypatch, mutant):
    """Plausible TLSF mistakes planted in the brute-force statement: taking
    the list that holds s' itself (no rounding up to a list bound), eight
    second-level lists instead of sixteen, and the first level alone (the
    segregated-fit class rule).  Each one fails a worked example."""
    from oracle import interval_ref as ir

    if mutant == "no_rounding":
        monkeypatch.setattr(ir, "_tlsf_fits", lambda lst, s: lst >= ir._tlsf_list(s))
    elif mutant == "eight_lists":
        monkeypatch.setattr(ir, "_tlsf_list",
                            lambda z: (ir._floor_log2(z), 2 * ((8 * (z - (1 << ir._floor_log2(z)))) >> ir._floor_log2(z))))
    else:
        monkeypatch.setattr(ir, "_tlsf_fits", lambda lst, s: 1 << lst[0] >= s)
    caught = False
    for case in load_tlsf_golden():
        a = ir.IntervalAllocator(case["arena"], case["min_block"], "tlsf")
        ok = True
        for frees, sizes, expect in case["batches"]:
            out, _ = a.batch(frees, sizes)
            ok &= [int(x) for x in out] == expect
        ok &= a.export_state() == case["final"]
        caught |= not ok
    assert caught, mutant


@pytest.mark.parametrize("seed", range(30))
def test_tlsf_oracle_equals_interval_allocator_random(seed):
    rng = np.random.default_rng(1000 + seed)
    mb = int(rng.choice([8, 16, 256]))
    A = mb * int(rng.integers(1, 400))
    o, r = oracle.Oracle(A, mb, "tlsf"), IntervalAllocator(A, mb, "tlsf")
    held = []
    for _ in range(80):
        nf = int(rng.integers(0, 4)) if held else 0
        frees = [held.pop(int(rng.integers(0, len(held)))) for _ in range(min(nf, len(held)))]
        if rng.random() < 0.3:
            frees.append(int(rng.integers(0, A // mb + 2)) * mb)  # often invalid
        sizes = [int(rng.integers(0, A // 2 + mb)) for _ in range(int(rng.integers(0, 5)))]
        oo, os_ = o.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        ro, rs = r.batch(frees, sizes)
        assert [int(x) for x in oo] == ro and [int(x) for x in os_] == rs
        held += [x for x in ro if x != FAIL and x not in held]
        held = [h for h in held if h not in frees or h in ro]
    assert [int(x) for x in o.export_state()] == r.export_state()


def test_tlsf_oracle_equals_interval_allocator_exhaustive():
    """Every sequence of up to four ops from a small alphabet on arenas of
    5, 12 and 31 granules: TLSF in both statements agrees op for op."""
    n = 0
    for G in (5, 12, 31):
        mb = 16
        alphabet = [("a", 16), ("a", 40), ("a", 100), ("a", 200), ("f", 0), ("f", 16), ("f", 48)]
        for seq in itertools.product(alphabet, repeat=4):
            o, r = oracle.Oracle(G * mb, mb, "tlsf"), IntervalAllocator(G * mb, mb, "tlsf")
            for kind, v in seq:
                if kind == "a":
                    assert o.malloc(v) == r.malloc(v)
                else:
                    assert o.free(v) == r.free(v)
            assert [int(x) for x in o.export_state()] == r.export_state()
            n += 1
    assert n == 3 * len(alphabet) ** 4


def test_tlsf_invariants_and_space_on_workload_traces():
    """Every intermediate TLSF state tiles the arena, never leaves two free
    blocks adjacent, keeps every free block in the list its size maps to,
    and its space report matches a walk of the blocks."""
    from paper_2405_07079_gb300 import workloads as W
    from oracle.interval_ref import _tlsf_list

    for wl in (W.tiny(n_ops=2000),
               W.Workload("l", 1 << 28, 512, lambda: W.Lifetimes(n_ops=30_000, batch=2048, mean_life=200)),
               W.usage(n_ops=1500, batch=8)):
        o = oracle.Oracle(wl.arena, wl.min_block, "tlsf")
        cl = wl.make()
        while (b := cl.next_batch()) is not None:
            out, st = o.batch(*b)
            cl.feed(out)
            s = oracle.decode_state(o.export_state(), "tlsf")
            blocks = s["blocks"]
            assert sum(sz for _, sz, _ in blocks) == s["arena"]
            assert all(not (a[2] and b2[2]) for a, b2 in zip(blocks, blocks[1:]))
            listed = {off: k for k, lst in enumerate(s["bins"]) for off in lst}
            free = {off: sz for off, sz, fr in blocks if fr}
            assert set(listed) == set(free)
            for off, k in listed.items():
                f, sl = _tlsf_list(free[off])
                assert k == 16 * f + sl
            for f in range(64):
                m = sum(1 << k for k in range(16) if s["bins"][16 * f + k])
                assert s["slmask"][f] == m and bool(s["bitmask"] >> f & 1) == bool(m)
            sp = o.space()
            assert sp["largest_free"] == max(free.values(), default=0)
            assert sp["extent"] == max([off + sz for off, sz, fr in blocks if not fr], default=0)


# ---- sequential fits on address-sorted lists (§3.1, §4) ---------------------
HAL_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hal_worked_examples.json")


def load_hal_golden():
    with open(HAL_GOLDEN) as f:
        doc = json.load(f)
    cases = []
    for c in doc["cases"]:
        fin = c["final"]
        w = [c["arena"], c["min_block"], len(fin["free"])]
        for a, z in fin["free"]:
            w += [a, z]
        w.append(len(fin["used"]))
        for a, z in fin["used"]:
            w += [a, z]
        w.append(fin["rover"])
        cases.append({"name": c["name"], "fit": c["fit"], "arena": c["arena"], "min_block": c["min_block"],
                      "batches": c["batches"], "final": w})
    return cases


def _hal_oracle(A, mb, fit):
    return oracle.HalOracle(A, mb, fit)


def _granule_fits(A, mb, fit):
    from oracle.fits_ref import GranuleFits

    return GranuleFits(A, mb, fit)


def _run_hal_case(a, case):
    ok = True
    for frees, sizes, expect, expect_st in case["batches"]:
        out, st = a.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        ok &= [int(x) for x in out] == expect and [int(x) for x in st] == expect_st
    return ok and [int(x) for x in a.export_state()] == case["final"]


@pytest.mark.parametrize("make", [_hal_oracle, _granule_fits])
@pytest.mark.parametrize("case", load_hal_golden(), ids=lambda c: c["name"].split()[0])
def test_hal_worked_example(make, case):
    a = make(case["arena"], case["min_block"], case["fit"])
    for frees, sizes, expect, expect_st in case["batches"]:
        out, st = a.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        assert [int(x) for x in out] == expect, case["name"]
        assert [int(x) for x in st] == expect_st, case["name"]
    assert [int(x) for x in a.export_state()] == case["final"], case["name"]


@pytest.mark.parametrize("mutant", ["best_ties_high", "next_no_wrap", "free_head", "next_from_start", "no_partial"])
def test_hal_worked_examples_catch_mutants(monkeypatch, mutant):
    """Plausible mistakes planted in the brute-force statement, each caught
    by a worked example: best fit preferring the higher address on a tie,
    next fit that does not wrap around, partial deallocation that frees the
    head of the block instead of its tail, next fit that ignores the rover,
    and a partial free that is rejected."""
    from oracle import fits_ref as fr

    cls = fr.GranuleFits
    if mutant == "best_ties_high":
        orig = cls.malloc

        def malloc(self, size):
            if self.fit != "best":
                return orig(self, size)
            s = -(-size // self.mb)
            fits = [r for r in self._runs() if r[1] >= s]
            if not size or not fits:
                return fr.FAIL
            start = min(fits, key=lambda r: (r[1], -r[0]))[0]
            for g in range(start, start + s):
                self.owner[g] = start
            self.size[start] = s
            self.rover = start + s
            return start * self.mb
        monkeypatch.setattr(cls, "malloc", malloc)
    elif mutant in ("next_no_wrap", "next_from_start"):
        orig_runs = cls._runs

        def runs(self):
            r = orig_runs(self)
            if self.fit == "next" and mutant == "next_no_wrap":
                return [x for x in r if x[0] + x[1] > self.rover] or r[:0]
            return r
        monkeypatch.setattr(cls, "_runs", runs)
        if mutant == "next_from_start":
            orig = cls.malloc

            def malloc(self, size):
                self.rover = 0
                return orig(self, size)
            monkeypatch.setattr(cls, "malloc", malloc)
    elif mutant == "free_head":
        def free(self, addr):
            if addr % self.mb or addr >= self.G * self.mb:
                return 1
            g = addr // self.mb
            b = self.owner[g]
            if b is None:
                return 1
            end = b + self.size[b]
            lo, hi = (b, g) if g != b else (b, end)
            for q in range(lo, hi):
                self.owner[q] = None
            if g == b:
                del self.size[b]
            else:
                for q in range(g, end):
                    self.owner[q] = g
                self.size[g] = end - g
                del self.size[b]
            return 0
        monkeypatch.setattr(cls, "free", free)
    else:
        orig = cls.free

        def free(self, addr):
            g = addr // self.mb if addr < self.G * self.mb else None
            if g is not None and self.owner[g] is not None and self.owner[g] != g:
                return 1
            return orig(self, addr)
        monkeypatch.setattr(cls, "free", free)
    caught = [not _run_hal_case(fr.GranuleFits(c["arena"], c["min_block"], c["fit"]), c) for c in load_hal_golden()]
    assert any(caught), mutant


@pytest.mark.parametrize("fit", ["first", "next", "best"])
@pytest.mark.parametrize("seed", range(12))
def test_hal_oracle_equals_granule_fits_random(fit, seed):
    from oracle.fits_ref import GranuleFits

    rng = np.random.default_rng(2000 + seed)
    mb = int(rng.choice([8, 16, 256]))
    A = mb * int(rng.integers(1, 120))
    o, r = oracle.HalOracle(A, mb, fit), GranuleFits(A, mb, fit)
    held = []
    for _ in range(60):
        frees = []
        for _ in range(int(rng.integers(0, 4))):
            if held and rng.random() < 0.7:
                a = held[int(rng.integers(0, len(held)))]
                # the start, or an interior granule (partial deallocation)
                frees.append(a + mb * int(rng.integers(0, 3)) if rng.random() < 0.4 else a)
            else:
                frees.append(int(rng.integers(0, A // mb + 2)) * mb + int(rng.choice([0, 0, 0, 3])))
        sizes = [int(rng.integers(0, A // 2 + mb)) for _ in range(int(rng.integers(0, 5)))]
        oo, os_ = o.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        ro, rs = r.batch(frees, sizes)
        assert [int(x) for x in oo] == ro and [int(x) for x in os_] == rs
        held = [a for a in held if a not in frees] + [x for x in ro if x != FAIL]
    assert [int(x) for x in o.export_state()] == r.export_state()


@pytest.mark.parametrize("fit", ["first", "next", "best"])
def test_hal_oracle_equals_granule_fits_exhaustive(fit):
    """Every sequence of four ops from a small alphabet (allocations of 1-3
    granules, frees of starts and interiors) on arenas of 4 and 9 granules."""
    from oracle.fits_ref import GranuleFits

    mb = 16
    alphabet = [("a", 16), ("a", 20), ("a", 48), ("f", 0), ("f", 16), ("f", 32), ("f", 40)]
    n = 0
    for G in (4, 9):
        for seq in itertools.product(alphabet, repeat=4):
            o, r = oracle.HalOracle(G * mb, mb, fit), GranuleFits(G * mb, mb, fit)
            for kind, v in seq:
                if kind == "a":
                    assert o.malloc(v) == r.malloc(v)
                else:
                    assert o.free(v) == r.free(v)
            assert [int(x) for x in o.export_state()] == r.export_state()
            n += 1
    assert n == 2 * len(alphabet) ** 4


@pytest.mark.parametrize("fit", ["first", "next", "best"])
def test_hal_invariants_on_workload_traces(fit):
    """After every batch: free and used blocks tile the arena without
    overlap, no two free blocks touch, sizes are multiples of min_block, and
    the counters match the lists."""
    from paper_2405_07079_gb300 import workloads as W

    for wl in (W.tiny(n_ops=2000), W.usage(n_ops=1500, batch=8),
               W.frag(n_fill=4000, n_big=400, batch=512, arena=32 << 20)):
        o = oracle.HalOracle(wl.arena, wl.min_block, fit)
        cl = wl.make()
        while (b := cl.next_batch()) is not None:
            out, st = o.batch(*b)
            cl.feed(out)
            s = oracle.decode_hal_state(o.export_state())
            blocks = sorted([(a, z, True) for a, z in s["free"]] + [(a, z, False) for a, z in s["used"]])
            pos = 0
            for a, z, fr in blocks:
                assert a == pos and z > 0 and a % wl.min_block == 0 and z % wl.min_block == 0
                pos = a + z
            assert pos == s["arena"]
            assert all(f1[0] + f1[1] < f2[0] for f1, f2 in zip(s["free"], s["free"][1:]))
            stt = o.stats()
            assert stt["used_bytes"] == sum(z for _, z in s["used"])
            assert stt["largest_free"] == max([z for _, z in s["free"]], default=0)
            assert stt["extent"] == max([a + z for a, z in s["used"]], default=0)


# ---- bitmask pool (§3.2) ----------------------------------------------------
BM_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bitmask_worked_examples.json")


def load_bitmask_golden():
    with open(BM_GOLDEN) as f:
        doc = json.load(f)
    cases = []
    for c in doc["cases"]:
        fin = c["final"]
        w = [c["pool"], c["unit"], len(fin["blocks"])]
        for a, z in fin["blocks"]:
            w += [a, z]
        w.append(fin["rover"])
        cases.append({"name": c["name"], "pool": c["pool"], "unit": c["unit"], "batches": c["batches"], "final": w})
    return cases


def _bm_oracle(P, u):
    return oracle.BitmaskOracle(P, u)


def _bm_ref(P, u):
    from oracle.fits_ref import BlockListPool

    return BlockListPool(P, u)


@pytest.mark.parametrize("make", [_bm_oracle, _bm_ref])
@pytest.mark.parametrize("case", load_bitmask_golden(), ids=lambda c: c["name"].split()[0])
def test_bitmask_worked_example(make, case):
    a = make(case["pool"], case["unit"])
    for frees, sizes, expect, expect_st in case["batches"]:
        out, st = a.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        assert [int(x) for x in out] == expect, case["name"]
        assert [int(x) for x in st] == expect_st, case["name"]
    assert [int(x) for x in a.export_state()] == case["final"], case["name"]


@pytest.mark.parametrize("mutant", ["first_fit", "runs_wrap", "free_to_next_free", "capped_at_64"])
def test_bitmask_worked_examples_catch_mutants(monkeypatch, mutant):
    """Plausible mistakes planted in the block-list statement, each caught
    by a worked example: first fit instead of next fit, runs that wrap past
    the pool's end, a free that releases units up to the next free unit
    (ignoring block starts), and objects capped at 64 units (one 128-bit
    window), which §3.2's 1 kB = 128-unit example rules out."""
    from oracle import fits_ref as fr

    cls = fr.BlockListPool
    if mutant == "first_fit":
        orig = cls.malloc

        def malloc(self, size):
            self.rover = 0
            return orig(self, size)
        monkeypatch.setattr(cls, "malloc", malloc)
    elif mutant == "runs_wrap":
        def free_at(self, p, k):
            units = [(p + j) % self.N for j in range(k)]
            return k <= self.N and all(not any(a <= q < a + n for a, n in self.blocks) for q in units)
        monkeypatch.setattr(cls, "_free_at", free_at)
    elif mutant == "free_to_next_free":
        orig = cls.free

        def free(self, addr):
            p = addr // self.unit
            blk = next((b for b in self.blocks if b[0] == p), None)
            r = orig(self, addr)
            if r == 0:  # also release the in-use blocks that follow, up to the next free unit
                q = p + blk[1]
                while (nxt := next((b for b in self.blocks if b[0] == q), None)) is not None:
                    self.blocks.remove(nxt)
                    q += nxt[1]
            return r
        monkeypatch.setattr(cls, "free", free)
    else:
        def malloc(self, size):  # runs capped at 64 units
            k = -(-size // self.unit) if size else 0
            if size == 0 or size > self.N * self.unit or k > 64 or k > self.N:
                return fr.FAIL
            order = list(range(self.rover, self.N)) + list(range(0, self.rover))
            p = next((q for q in order if self._free_at(q, k)), None)
            if p is None:
                return fr.FAIL
            self.blocks.append((p, k))
            self.rover = p + k
            return p * self.unit
        monkeypatch.setattr(cls, "malloc", malloc)
    caught = False
    for c in load_bitmask_golden():
        a = cls(c["pool"], c["unit"])
        ok = True
        for frees, sizes, expect, expect_st in c["batches"]:
            out, st = a.batch(frees, sizes)
            ok &= [int(x) for x in out] == expect and [int(x) for x in st] == expect_st
        ok &= a.export_state() == c["final"]
        caught |= not ok
    assert caught, mutant


@pytest.mark.parametrize("seed", range(20))
def test_bitmask_oracle_equals_block_list_random(seed):
    from oracle.fits_ref import BlockListPool

    rng = np.random.default_rng(3000 + seed)
    u = int(rng.choice([8, 16, 64]))
    N = int(rng.integers(1, 400))
    o, r = oracle.BitmaskOracle(N * u, u), BlockListPool(N * u, u)
    held = []
    for _ in range(60):
        frees = []
        for _ in range(int(rng.integers(0, 5))):
            if held and rng.random() < 0.75:
                h = held[int(rng.integers(0, len(held)))]
                frees.append(h + (u if rng.random() < 0.15 else 0))
            else:
                frees.append(int(rng.integers(0, N + 3)) * u + int(rng.choice([0, 0, 4])))
        sizes = [int(rng.integers(0, (min(N, 70) if rng.random() < 0.7 else N) * u + 2))
                 for _ in range(int(rng.integers(0, 6)))]
        oo, os_ = o.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
        ro, rs = r.batch(frees, sizes)
        assert [int(x) for x in oo] == ro and [int(x) for x in os_] == rs
        held = [h for h in held if h not in frees] + [x for x in ro if x != FAIL]
    assert [int(x) for x in o.export_state()] == r.export_state()


@pytest.mark.parametrize("seed", range(12))
def test_bitmask_frees_commute(seed):
    """The frees of one batch commute: applied in any order they leave the
    same pool, and the free statuses move with the frees, except that among
    frees of one block the first in the order applied succeeds.  (A free
    only turns a marked block start into free units, so no free moves the
    end of another block; the GPU resolves a batch's frees at once on this
    property.)  Checked on the oracle by replaying one pool's history and then
    one free batch in its order and in a shuffled order."""
    rng = np.random.default_rng(7100 + seed)
    u = 8
    N = int(rng.integers(64, 3000))
    hist = []
    o = oracle.BitmaskOracle(N * u, u)
    held = []
    for _ in range(12):  # a fragmented pool: objects of 1-80 units, some freed
        fr = [held[int(i)] for i in rng.choice(len(held), len(held) // 3, replace=False)] if held else []
        sz = (rng.integers(1, 80, int(rng.integers(5, 60))) * u).tolist()
        out, _ = o.batch(np.array(fr, np.uint64), np.array(sz, np.uint64))
        hist.append((fr, sz))
        held = [h for h in held if h not in fr] + [int(x) for x in out if x != FAIL]
    frees = [held[int(i)] for i in rng.choice(len(held), min(len(held), 40), replace=False)]
    frees += [frees[int(i)] for i in rng.integers(0, len(frees), 8)]          # the same block twice
    frees += [h + u for h in frees[:5]] + [int(rng.integers(0, N + 2)) * u]    # interior, anywhere
    perm = rng.permutation(len(frees))

    def run(order):
        p = oracle.BitmaskOracle(N * u, u)
        for fr, sz in hist:
            p.batch(np.array(fr, np.uint64), np.array(sz, np.uint64))
        _, st = p.batch(np.array(order, np.uint64), np.array([], np.uint64))
        return p.export_state(), [int(x) for x in st]

    s1, st1 = run(frees)
    s2, st2 = run([frees[i] for i in perm])
    assert np.array_equal(s1, s2)
    assert sum(1 for x in st1 if x == 0) == sum(1 for x in st2 if x == 0)
    ok1 = {frees[i] for i, x in enumerate(st1) if x == 0}
    ok2 = {frees[perm[i]] for i, x in enumerate(st2) if x == 0}
    assert ok1 == ok2 and len(ok1) >= 10


def test_bitmask_oracle_equals_block_list_exhaustive():
    """Every sequence of four ops from a small alphabet on pools of 3 and 7
    units."""
    from oracle.fits_ref import BlockListPool

    alphabet = [("a", 8), ("a", 16), ("a", 20), ("f", 0), ("f", 8), ("f", 16), ("f", 4)]
    n = 0
    for N in (3, 7):
        for seq in itertools.product(alphabet, repeat=4):
            o, r = oracle.BitmaskOracle(N * 8, 8), BlockListPool(N * 8, 8)
            for kind, v in seq:
                if kind == "a":
                    assert o.malloc(v) == r.malloc(v)
                else:
                    assert o.free(v) == r.free(v)
            assert [int(x) for x in o.export_state()] == r.export_state()
            n += 1
    assert n == 2 * len(alphabet) ** 4


def test_property_hypothesis():
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    op = st.one_of(st.tuples(st.just("a"), st.integers(0, 600)),
                   st.tuples(st.just("f"), st.integers(0, 40).map(lambda g: g * 16)))

    @hyp.settings(max_examples=300, deadline=None)
    @hyp.given(st.lists(st.lists(op, max_size=6), max_size=12))
    def prop(batches):
        A, mb = 512, 16
        o, r = oracle.Oracle(A, mb), IntervalAllocator(A, mb)
        for b in batches:
            frees = [v for k, v in b if k == "f"]
            sizes = [v for k, v in b if k == "a"]
            oo, os_ = o.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
            ro, rs = r.batch(frees, sizes)
            assert [int(x) for x in oo] == ro and [int(x) for x in os_] == rs
            check_invariants(o.export_state())
        assert [int(x) for x in o.export_state()] == r.export_state()

    prop()


def test_property_hypothesis_other_policies():
    """Random op sequences (hypothesis) for TLSF, the three sequential fits
    (frees of starts and interior granules) and the bitmask pool: each oracle
    equals its independent restatement op for op and in its final state."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    from oracle.fits_ref import BlockListPool, GranuleFits

    op = st.one_of(st.tuples(st.just("a"), st.integers(0, 600)),
                   st.tuples(st.just("f"), st.integers(0, 40).map(lambda g: g * 16)),
                   st.tuples(st.just("f"), st.integers(0, 700)))

    def pair_run(o, r, batches):
        for b in batches:
            frees = [v for k, v in b if k == "f"]
            sizes = [v for k, v in b if k == "a"]
            oo, os_ = o.batch(np.array(frees, np.uint64), np.array(sizes, np.uint64))
            ro, rs = r.batch(frees, sizes)
            assert [int(x) for x in oo] == list(ro) and [int(x) for x in os_] == list(rs)
        assert [int(x) for x in o.export_state()] == r.export_state()

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(st.lists(st.lists(op, max_size=6), max_size=10))
    def prop(batches):
        A, mb = 512, 16
        pair_run(oracle.Oracle(A, mb, "tlsf"), IntervalAllocator(A, mb, "tlsf"), batches)
        for fit in ("first", "next", "best"):
            pair_run(oracle.HalOracle(A, mb, fit), GranuleFits(A, mb, fit), batches)
        pair_run(oracle.BitmaskOracle(A, 8), BlockListPool(A, 8), batches)

    prop()
