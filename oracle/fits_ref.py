"""Brute-force restatement of the sequential fits (§3.1 Algorithms 1 and 2, §4
Algorithm 3 and the first/next-fit variants) on tiny arenas.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A different formulation from ``hal_oracle.c`` so that the two pin each
other:

* The heap is a map from granule to owner: ``None`` for a free granule, else
  the start of the in-use block that holds it.  There is no free list: the
  free blocks are the maximal runs of free granules, recomputed for every
  request, so coalescing never has to be written down.
* First fit takes the first run (in address order) at least s' long; best
  fit the shortest such run, the lowest address among equal lengths; next
  fit the first such run in address order starting from the run that
  contains or follows the rover, wrapping around.
* Freeing an address inside an in-use block frees the granules from that
  address to the block's end (the whole block when it is the start).

Pure-Python loops: for arenas of a few dozen granules and short traces only.
"""
from __future__ import annotations

FAIL = 0xFFFFFFFFFFFFFFFF


class GranuleFits:
    def __init__(self, arena_bytes: int, min_block: int, fit: str = "first"):
        assert min_block >= 8 and min_block & (min_block - 1) == 0 and fit in ("first", "next", "best")
        self.mb = min_block
        self.G = arena_bytes // min_block
        assert self.G > 0
        self.fit = fit
        self.owner = [None] * self.G
        self.size = {}   # block start granule -> granules
        self.rover = 0   # granules

    def _runs(self):
        runs, g = [], 0
        while g < self.G:
            if self.owner[g] is None:
                h = g
                while g < self.G and self.owner[g] is None:
                    g += 1
                runs.append((h, g - h))
            else:
                g += 1
        return runs

    def malloc(self, size: int) -> int:
        if size == 0 or size > self.G * self.mb:
            return FAIL
        s = -(-size // self.mb)
        runs = [r for r in self._runs()]
        fits = [r for r in runs if r[1] >= s]
        if not fits:
            return FAIL
        if self.fit == "first":
            start = fits[0][0]
        elif self.fit == "best":
            start = min(fits, key=lambda r: (r[1], r[0]))[0]
        else:
            k0 = next((k for k, r in enumerate(runs) if r[0] + r[1] > self.rover), len(runs))
            order = runs[k0:] + runs[:k0]
            start = next(r for r in order if r[1] >= s)[0]
        for g in range(start, start + s):
            self.owner[g] = start
        self.size[start] = s
        self.rover = start + s
        return start * self.mb

    def free(self, addr: int) -> int:
        if addr % self.mb or addr >= self.G * self.mb:
            return 1
        g = addr // self.mb
        b = self.owner[g]
        if b is None:
            return 1
        end = b + self.size[b]
        for q in range(g, end):
            self.owner[q] = None
        if g == b:
            del self.size[b]
        else:
            self.size[b] = g - b
        return 0

    def batch(self, frees, sizes):
        st = [self.free(int(a)) for a in frees]
        out = [self.malloc(int(s)) for s in sizes]
        return out, st

    def export_state(self) -> list:
        """The oracle's canonical words: free runs, used blocks, rover."""
        mb = self.mb
        runs = self._runs()
        w = [self.G * mb, mb, len(runs)]
        for h, n in runs:
            w += [h * mb, n * mb]
        used = sorted(self.size.items())
        w.append(len(used))
        for b, n in used:
            w += [b * mb, n * mb]
        return w + [self.rover * mb]


class BlockListPool:
    """The bitmask pool (§3.2) restated without bits: the in-use blocks are
    a list of (first unit, units) intervals; a unit is free iff no interval
    covers it.  Next fit over candidate starts: the lowest start at or after
    the rover whose k units are all free, else the lowest start of all.  A
    free must name the first unit of a listed block and removes it.  The
    second bitmap of the C oracle is the list's set of starts."""

    def __init__(self, pool_bytes: int, unit: int):
        self.unit = unit
        self.N = pool_bytes // unit
        self.blocks = []  # (first unit, units), in allocation order
        self.rover = 0

    def _free_at(self, p, k):
        return p + k <= self.N and all(not (a < p + k and p < a + n) for a, n in self.blocks)

    def malloc(self, size: int) -> int:
        k = -(-size // self.unit) if size else 0
        if size == 0 or size > self.N * self.unit or k > self.N:
            return FAIL
        order = list(range(self.rover, self.N)) + list(range(0, self.rover))
        p = next((q for q in order if self._free_at(q, k)), None)
        if p is None:
            return FAIL
        self.blocks.append((p, k))
        self.rover = p + k
        return p * self.unit

    def free(self, addr: int) -> int:
        if addr % self.unit:
            return 1
        p = addr // self.unit
        for i, (a, n) in enumerate(self.blocks):
            if a == p:
                del self.blocks[i]
                return 0
        return 1

    def batch(self, frees, sizes):
        st = [self.free(int(a)) for a in frees]
        out = [self.malloc(int(s)) for s in sizes]
        return out, st

    def export_state(self) -> list:
        w = [self.N * self.unit, self.unit, len(self.blocks)]
        for a, n in sorted(self.blocks):
            w += [a * self.unit, n * self.unit]
        return w + [self.rover * self.unit]
