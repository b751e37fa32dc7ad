"""Brute-force restatement of the segregated-fit policy (§5.1) on tiny arenas.

TEST INFRASTRUCTURE ONLY (see the package docstring).

This is deliberately a different formulation from ``segfit_oracle.c`` so the
two pin each other:

* The heap is a Python list of intervals ``[start, size, free, stamp]`` kept
  in address order; there are no linked lists, no bitmap and no prev_adj.
* Every push onto a free list (Algorithm 4's split remainder, Algorithm 5's
  final push) is replaced by giving the block a fresh, strictly increasing
  stamp.  A LIFO list is therefore "its members by decreasing stamp", and its
  head is the member with the largest stamp.
* Allocation: round up to min_block, take the class c = ceil(log2 s'); among
  free intervals whose floor(log2 size) >= c, the lowest such class wins and
  inside it the largest stamp wins; the front s' bytes become used and the
  rest, if any, is a new free interval with a fresh stamp.
* Free: the interval must start exactly at the address and be in use; it
  becomes free, merges with free neighbours on both sides (found by scanning
  the ordered list), and the merged interval gets a fresh stamp.

Two-level segregated fit (§5.2, ``policy="tlsf"``) in the same terms: the
list of a free interval of size z is (f, k) with f = floor(log2 z) and
k = floor(16 (z - 2^f) / 2^f), i.e. the sixteenth of [2^f, 2^(f+1)) that z
falls in; the list's lower bound is (16 + k) 2^f / 16.  An allocation of s'
may take a list whose lower bound is >= s' (then all of its members fit);
the lowest such list wins, and inside it the largest stamp.  The oracle finds
that list with bit masks and a rounding trick instead; this statement uses
the bounds themselves.

Pure-Python loops: for arenas of a few dozen granules and short traces only.
"""
from __future__ import annotations

FAIL = 0xFFFFFFFFFFFFFFFF


def _floor_log2(x: int) -> int:
    return x.bit_length() - 1


def _ceil_log2(x: int) -> int:
    return (x - 1).bit_length() if x > 1 else 0


def _tlsf_list(z: int):
    f = _floor_log2(z)
    return f, (16 * (z - (1 << f))) >> f


def _tlsf_fits(lst, s: int) -> bool:
    f, k = lst
    return (16 + k) << f >= 16 * s


class IntervalAllocator:
    def __init__(self, arena_bytes: int, min_block: int, policy: str = "segfit"):
        assert min_block >= 8 and min_block & (min_block - 1) == 0
        assert policy in ("segfit", "tlsf")
        self.policy = policy
        self.arena = arena_bytes - arena_bytes % min_block
        assert self.arena > 0
        self.min_block = min_block
        self.clock = 0
        self.iv = [[0, self.arena, True, self._tick()]]

    def _tick(self) -> int:
        self.clock += 1
        return self.clock

    def malloc(self, size: int) -> int:
        if size == 0 or size > self.arena:
            return FAIL
        s = -(-size // self.min_block) * self.min_block
        if s > self.arena:
            return FAIL
        c = _ceil_log2(s)
        best = None
        for k, (st, sz, fr, stamp) in enumerate(self.iv):
            if not fr:
                continue
            if self.policy == "tlsf":
                lst = _tlsf_list(sz)
                if not _tlsf_fits(lst, s):
                    continue
                key = (lst, -stamp)
            else:
                if _floor_log2(sz) < c:
                    continue
                key = (_floor_log2(sz), -stamp)
            if best is None or key < best[0]:
                best = (key, k)
        if best is None:
            return FAIL
        k = best[1]
        st, sz, _, _ = self.iv[k]
        self.iv[k] = [st, s, False, 0]
        if sz > s:
            self.iv.insert(k + 1, [st + s, sz - s, True, self._tick()])
        return st

    def free(self, addr: int) -> int:
        k = next((i for i, v in enumerate(self.iv) if v[0] == addr), None)
        if k is None or self.iv[k][2]:
            return 1
        lo, hi = k, k
        if k > 0 and self.iv[k - 1][2]:
            lo = k - 1
        if k + 1 < len(self.iv) and self.iv[k + 1][2]:
            hi = k + 1
        start = self.iv[lo][0]
        size = sum(v[1] for v in self.iv[lo:hi + 1])
        self.iv[lo:hi + 1] = [[start, size, True, self._tick()]]
        return 0

    def batch(self, frees, sizes):
        st = [self.free(int(a)) for a in frees]
        out = [self.malloc(int(s)) for s in sizes]
        return out, st

    def export_state(self) -> list:
        """Same canonical words as the C oracle (blocks, bins by stamp, bitmap;
        TLSF: the 64 x 16 lists, the first-level and second-level masks)."""
        w = [self.arena, self.min_block, len(self.iv)]
        for st, sz, fr, _ in self.iv:
            w += [st, sz | (int(fr) << 63)]
        if self.policy == "tlsf":
            fl, sl = 0, [0] * 64
            for f in range(64):
                for k in range(16):
                    members = sorted((v for v in self.iv if v[2] and _tlsf_list(v[1]) == (f, k)),
                                     key=lambda v: -v[3])
                    w.append(len(members))
                    w += [v[0] for v in members]
                    if members:
                        fl |= 1 << f
                        sl[f] |= 1 << k
            return w + [fl] + sl
        bitmask = 0
        for b in range(64):
            members = sorted((v for v in self.iv if v[2] and _floor_log2(v[1]) == b),
                             key=lambda v: -v[3])
            w.append(len(members))
            w += [v[0] for v in members]
            if members:
                bitmask |= 1 << b
        w.append(bitmask)
        return w
