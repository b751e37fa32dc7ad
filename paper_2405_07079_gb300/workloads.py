"""Seeded synthetic request streams for the allocator.

This module is the one piece shared by the GPU path and the CPU oracle.  It
holds none of the allocator's arithmetic: no rounding, no size classes, no
placement.  A generator plays the *client* of an allocator -- it decides
which sizes to request and which of the offsets it currently holds to give
back -- and it learns what it holds only from the results it is fed.  Run in
lock step with any allocator it yields a concrete trace (per batch: a list of
offsets to free and a list of sizes to allocate); two exact allocators fed by
two instances of the same generator produce the same trace.

The paper measures on the malloc-large benchmark of mimalloc-bench (§6):
random allocations and frees of 1 kB to 16 MB blocks.  That benchmark is not
reproduced; the streams below are synthetic stand-ins whose size ranges
cover it.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``(seed, field)`` is
``mix(key(seed, field) + (i + 1) * 0x9E3779B97F4A7C15)``.  Every draw is
indexed by the op slot it belongs to, so the draws themselves never depend
on allocator results.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
FAIL = 0xFFFFFFFFFFFFFFFF
BASE_SEED = 2405070790

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based splitmix64 stream keyed by (seed, field name)."""

    def __init__(self, seed: int, name: str):
        tag = np.uint64(sum((b + 1) << (8 * (i % 8)) for i, b in enumerate(name.encode())) & (2**64 - 1))
        with np.errstate(over="ignore"):
            self.key = _mix(np.array([np.uint64(seed) ^ tag], dtype=np.uint64))[0]

    def u64(self, idx) -> np.ndarray:
        i = np.asarray(idx, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return _mix(self.key + (i + np.uint64(1)) * GAMMA)

    def unif(self, idx) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def log_uniform(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """floor(exp(ln lo + u (ln hi - ln lo))), clamped to [lo, hi]."""
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))
    return np.clip(v, lo, hi).astype(np.uint64)


def tensor_mix(u_mix: np.ndarray, u_size: np.ndarray) -> np.ndarray:
    """70 % powers of two 2^U{12..21} (4 KiB..2 MiB), 30 % log-uniform 256 B..256 MiB."""
    pow2 = np.left_shift(np.uint64(1), (12 + np.minimum(np.floor(u_size * 10), 9)).astype(np.uint64))
    lu = log_uniform(u_size, 256, 256 * MiB)
    return np.where(u_mix < 0.7, pow2, lu).astype(np.uint64)


def geometric(u: np.ndarray, mean: float) -> np.ndarray:
    """Geometric lifetimes on {1, 2, ...} with success probability 1/mean."""
    p = 1.0 / mean
    return (1 + np.floor(np.log1p(-u) / math.log1p(-p))).astype(np.int64)


# --------------------------------------------------------------------------
# Closed-loop clients.  Protocol: ``b = next_batch()`` returns
# ``(frees uint64[], sizes uint64[])`` or ``None`` at the end; ``feed(out)``
# hands back the offsets the allocator returned for ``sizes``.
# --------------------------------------------------------------------------


class TinyRandom:
    """Small random trace: per op, a free with probability ``p_free`` when a
    pre-batch live allocation is not yet targeted in this batch (target uniform
    over those), else a malloc of a log-uniform size."""

    def __init__(self, n_ops=10_000, batch=64, p_free=0.4, lo=256, hi=64 * KiB, seed=BASE_SEED + 1):
        self.n_ops, self.bs, self.p_free, self.lo, self.hi = n_ops, batch, p_free, lo, hi
        self.s_type, self.s_pick, self.s_size = (Stream(seed, f) for f in ("type", "pick", "size"))
        self.t = 0
        self.live: list[int] = []  # offsets held, in order of allocation
        self._pending_free: set[int] = set()

    def next_batch(self):
        if self.t >= self.n_ops:
            return None
        n = min(self.bs, self.n_ops - self.t)
        idx = np.arange(self.t, self.t + n)
        ut, up = self.s_type.unif(idx), self.s_pick.unif(idx)
        sz = log_uniform(self.s_size.unif(idx), self.lo, self.hi)
        cand = list(self.live)
        frees, sizes = [], []
        for k in range(n):
            if ut[k] < self.p_free and cand:
                j = int(up[k] * len(cand))
                frees.append(cand[j])
                cand[j] = cand[-1]
                cand.pop()
            else:
                sizes.append(int(sz[k]))
        self.t += n
        self._pending_free = set(frees)
        return np.array(frees, dtype=np.uint64), np.array(sizes, dtype=np.uint64)

    def feed(self, out):
        self.live = [a for a in self.live if a not in self._pending_free]
        self.live += [int(a) for a in out if int(a) != FAIL]


class Lifetimes:
    """Large trace: each op slot emits a due free if one exists, else a malloc
    (tensor-like size mix); lifetimes are geometric in ops.  A free that falls
    due inside its own allocation's batch is deferred to the first slot of the
    next batch."""

    def __init__(self, n_ops=10_000_000, batch=65_536, mean_life=1000.0, seed=BASE_SEED + 2,
                 scale=1.0, min_size=0):
        self.n_ops, self.bs, self.mean_life, self.scale, self.min_size = n_ops, batch, mean_life, scale, min_size
        self.s_mix, self.s_size, self.s_life = (Stream(seed, f) for f in ("mix", "size", "life"))
        self.t = 0
        # pending frees: due slot, allocation slot (tie-break), offset
        self.p_due = np.zeros(0, np.int64)
        self.p_seq = np.zeros(0, np.int64)
        self.p_off = np.zeros(0, np.uint64)
        self._last = None

    def _sizes(self, idx):
        s = tensor_mix(self.s_mix.unif(idx), self.s_size.unif(idx))
        if self.scale != 1.0:
            s = np.floor(s.astype(np.float64) * self.scale).astype(np.uint64)
        if self.min_size:
            s = np.maximum(s, np.uint64(self.min_size))
        return s

    def next_batch(self):
        if self.t >= self.n_ops:
            return None
        n = min(self.bs, self.n_ops - self.t)
        T0 = self.t
        order = np.lexsort((self.p_seq, self.p_due))
        d = self.p_due[order] - T0
        k = np.arange(d.size)
        slot = np.maximum.accumulate(np.maximum(d - k, 0)) + k if d.size else d
        emit = order[slot < n]
        free_slots = slot[slot < n]
        is_free = np.zeros(n, bool)
        is_free[free_slots] = True
        frees = self.p_off[emit]
        keep = np.ones(self.p_due.size, bool)
        keep[emit] = False
        self.p_due, self.p_seq, self.p_off = self.p_due[keep], self.p_seq[keep], self.p_off[keep]
        m_slots = np.nonzero(~is_free)[0] + T0
        sizes = self._sizes(m_slots)
        life = geometric(self.s_life.unif(m_slots), self.mean_life)
        self._last = (m_slots, life, T0 + n)
        self.t += n
        return frees.astype(np.uint64), sizes

    def feed(self, out):
        m_slots, life, end = self._last
        out = np.asarray(out, dtype=np.uint64)
        ok = out != np.uint64(FAIL)
        due = np.maximum(m_slots[ok] + life[ok], end)
        self.p_due = np.concatenate([self.p_due, due])
        self.p_seq = np.concatenate([self.p_seq, m_slots[ok]])
        self.p_off = np.concatenate([self.p_off, out[ok]])

    def live_count(self) -> int:
        return int(self.p_off.size)


class FragStress:
    """Fill with n_fill allocations of 4 KiB, free every other one (indices
    0, 2, 4, ... ascending), request n_big log-uniform 8 KiB..64 MiB, then free
    everything still held in a seeded random order.  Batches of ``batch``."""

    def __init__(self, n_fill=1_000_000, n_big=50_000, batch=16_384, fill_size=4 * KiB,
                 big_lo=8 * KiB, big_hi=64 * MiB, seed=BASE_SEED + 3):
        self.n_fill, self.n_big, self.bs, self.fill_size = n_fill, n_big, batch, fill_size
        self.big_lo, self.big_hi = big_lo, big_hi
        self.s_size, self.s_perm = Stream(seed, "size"), Stream(seed, "perm")
        self.phase, self.pos = "fill", 0
        self.fill_out: list[np.ndarray] = []
        self.big_out: list[np.ndarray] = []
        self._targets = None
        self._expect = None

    def next_batch(self):
        e64 = np.zeros(0, np.uint64)
        if self.phase == "fill":
            n = min(self.bs, self.n_fill - self.pos)
            self._expect = "fill"
            self.pos += n
            if self.pos >= self.n_fill:
                self.phase, self.pos = "free_even", 0
            return e64, np.full(n, self.fill_size, np.uint64)
        if self.phase == "free_even":
            if self._targets is None:
                fo = np.concatenate(self.fill_out) if self.fill_out else e64
                self._held_fill = fo
                self._targets = fo[0::2][fo[0::2] != np.uint64(FAIL)]
            t = self._targets[self.pos:self.pos + self.bs]
            self.pos += t.size
            self._expect = None
            if self.pos >= self._targets.size:
                self.phase, self.pos, self._targets = "big", 0, None
            return t, e64
        if self.phase == "big":
            n = min(self.bs, self.n_big - self.pos)
            idx = np.arange(self.pos, self.pos + n)
            self.pos += n
            self._expect = "big"
            if self.pos >= self.n_big:
                self.phase, self.pos = "free_all", 0
            return e64, log_uniform(self.s_size.unif(idx), self.big_lo, self.big_hi)
        if self.phase == "free_all":
            if self._targets is None:
                odd = self._held_fill[1::2]
                big = np.concatenate(self.big_out) if self.big_out else e64
                held = np.concatenate([odd, big])
                held = held[held != np.uint64(FAIL)]
                keys = self.s_perm.u64(np.arange(held.size))
                self._targets = held[np.argsort(keys, kind="stable")]
            t = self._targets[self.pos:self.pos + self.bs]
            self.pos += t.size
            self._expect = None
            if self.pos >= self._targets.size:
                self.phase = "done"
            return t, e64
        return None

    def feed(self, out):
        if self._expect == "fill":
            self.fill_out.append(np.asarray(out, np.uint64).copy())
        elif self._expect == "big":
            self.big_out.append(np.asarray(out, np.uint64).copy())


class MultiLifetimes:
    """Many independent arenas, one batch for all of them per step (CSR).

    Per arena and batch: n ~ U{0..max_ops} request slots; the frees due by the
    end of the slots come first (earliest due first, at most n), the remaining
    slots are mallocs with the large-trace size mix scaled by the arena's size
    (clamped to >= min_size); lifetimes are geometric in the arena's own op
    count.  A free falling due inside its allocation's own batch waits for the
    next batch.  Vectorised over arenas: the pending frees of all arenas live
    in one sorted array of keys ``arena << 49 | due << 30 | seq``.
    """

    def __init__(self, arena_bytes, n_batches=200, max_ops=2048, mean_life=1000.0, min_size=256,
                 seed=BASE_SEED + 4, ref_bytes=16 * GiB):
        self.A = np.asarray(arena_bytes, dtype=np.uint64)
        self.na = self.A.size
        assert self.na < (1 << 15)
        self.nb, self.max_ops, self.mean_life, self.min_size = n_batches, max_ops, mean_life, min_size
        self.scale = self.A.astype(np.float64) / float(ref_bytes)
        self.s_n, self.s_mix, self.s_size, self.s_life = (Stream(seed, f) for f in ("n", "mix", "size", "life"))
        self.b = 0
        self.t = np.zeros(self.na, np.int64)          # per-arena op clock
        self.keys = np.zeros(0, np.uint64)             # pending frees, sorted
        self.offs = np.zeros(0, np.uint64)
        self.seq = 0
        self._last = None
        self._ids = np.arange(self.na, dtype=np.uint64)

    def next_batch(self):
        """Returns (free_rowptr uint32[n+1], frees uint64[], alloc_rowptr uint32[n+1], sizes uint64[])."""
        if self.b >= self.nb:
            return None
        ids = self._ids
        n = np.floor(self.s_n.unif(np.uint64(self.b) * np.uint64(self.na) + ids) * (self.max_ops + 1)).astype(np.int64)
        hi = (ids << np.uint64(49)) | ((self.t + n).astype(np.uint64) << np.uint64(30))
        seg = np.searchsorted(self.keys, ids << np.uint64(49))
        elig = np.searchsorted(self.keys, hi) - seg
        f = np.minimum(elig, n)
        fsum = int(f.sum())
        first = np.cumsum(f) - f
        idx = np.repeat(seg, f) + (np.arange(fsum) - np.repeat(first, f))
        frees = self.offs[idx]
        keep = np.ones(self.keys.size, bool)
        keep[idx] = False
        self.keys, self.offs = self.keys[keep], self.offs[keep]
        m = n - f
        msum = int(m.sum())
        marena = np.repeat(np.arange(self.na), m)
        mstart = np.cumsum(m) - m
        k = np.arange(msum) - np.repeat(mstart, m)
        slot = np.repeat(self.t + f, m) + k                       # arena op index of each malloc
        draw = marena.astype(np.uint64) * np.uint64(1 << 24) + slot.astype(np.uint64)
        sz = tensor_mix(self.s_mix.unif(draw), self.s_size.unif(draw)).astype(np.float64)
        sz = np.maximum(np.floor(sz * self.scale[marena]), self.min_size).astype(np.uint64)
        life = geometric(self.s_life.unif(draw), self.mean_life)
        self._last = (marena, slot, life, self.t + n)
        self.t = self.t + n
        self.b += 1
        frow = np.concatenate([[0], np.cumsum(f)]).astype(np.uint32)
        arow = np.concatenate([[0], np.cumsum(m)]).astype(np.uint32)
        return frow, frees.astype(np.uint64), arow, sz

    def feed(self, out):
        marena, slot, life, end = self._last
        out = np.asarray(out, np.uint64)
        ok = out != np.uint64(FAIL)
        a = marena[ok]
        due = np.maximum(slot[ok] + life[ok], end[a])
        seq = self.seq + np.arange(a.size, dtype=np.int64)
        self.seq += a.size
        nk = (a.astype(np.uint64) << np.uint64(49)) | (due.astype(np.uint64) << np.uint64(30)) | seq.astype(np.uint64)
        order = np.argsort(nk, kind="stable")
        nk, no = nk[order], out[ok][order]
        pos = np.searchsorted(self.keys, nk)
        self.keys = np.insert(self.keys, pos, nk)
        self.offs = np.insert(self.offs, pos, no)


class RandomSlots:
    """The malloc-large pattern as §6 describes it, as a client: ``slots``
    slots, and per op a slot drawn uniformly; a slot that holds a block has
    it freed, an empty one gets a malloc of a log-uniform size in
    ``[lo, hi]`` (1 kB to 16 MB by default; a failed malloc leaves the slot
    empty).  Ops are cut into batches of at most ``batch`` ops in which every
    free comes before every malloc and no slot appears twice, so that the
    batched trace applies the ops in their sequential order."""

    def __init__(self, n_ops=5000, slots=64, lo=1 * KiB, hi=16 * MiB, batch=1, seed=BASE_SEED + 6):
        self.n_ops, self.slots, self.lo, self.hi, self.bs = n_ops, slots, lo, hi, batch
        self.s_pick, self.s_size = Stream(seed, "slot"), Stream(seed, "size")
        self.held: list[int | None] = [None] * slots
        self.t = 0
        self._filling: list[int] = []

    def next_batch(self):
        if self.t >= self.n_ops:
            return None
        frees, sizes, touched = [], [], set()
        self._filling = []
        while self.t < self.n_ops and len(frees) + len(sizes) < self.bs:
            j = min(int(self.s_pick.unif([self.t])[0] * self.slots), self.slots - 1)
            held = self.held[j]
            if j in touched or (held is not None and sizes):
                break  # the op would break sequential order: it starts the next batch
            touched.add(j)
            if held is not None:
                frees.append(held)
                self.held[j] = None
            else:
                sizes.append(int(log_uniform(self.s_size.unif([self.t]), self.lo, self.hi)[0]))
                self._filling.append(j)
            self.t += 1
        return np.array(frees, dtype=np.uint64), np.array(sizes, dtype=np.uint64)

    def feed(self, out):
        for j, off in zip(self._filling, np.asarray(out).tolist()):
            if off != FAIL:
                self.held[j] = int(off)


def serving_arrivals(lam: float, seconds: float, page=16 * KiB, max_pages=512, hold_mean_ns=20e6,
                     seed=BASE_SEED + 5):
    """Open-loop requests: Poisson arrivals at ``lam`` per second for
    ``seconds``; each a malloc of U{1..max_pages} pages held for an
    exponential time (mean ``hold_mean_ns``), then freed.  uint64[n, 3]:
    arrival ns, bytes, hold ns."""
    n = int(lam * seconds * 1.1) + 16
    idx = np.arange(n)
    gaps = -np.log1p(-Stream(seed, "gap").unif(idx)) / lam * 1e9
    t = np.floor(np.cumsum(gaps)).astype(np.uint64)
    keep = t < np.uint64(seconds * 1e9)
    t = t[keep]
    m = t.size
    pages = 1 + np.floor(Stream(seed, "pages").unif(idx[:m]) * max_pages).astype(np.uint64)
    hold = np.floor(-np.log1p(-Stream(seed, "hold").unif(idx[:m])) * hold_mean_ns).astype(np.uint64)
    return np.stack([t, pages * np.uint64(page), np.maximum(hold, 1)], axis=1).astype(np.uint64)


def multi_arena_sizes(n_arenas=4096, lo=64 * MiB, hi=1 * GiB, granule=256, seed=BASE_SEED + 4):
    """Arena sizes log-uniform in [lo, hi], rounded down to the granule."""
    s = log_uniform(Stream(seed, "arena").unif(np.arange(n_arenas)), lo, hi)
    return (s // np.uint64(granule)) * np.uint64(granule)


# --------------------------------------------------------------------------
# Named workloads (sizes of the five synthetic configurations)
# --------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    arena: int
    min_block: int
    make: object               # () -> client
    note: str = ""
    extra: dict = field(default_factory=dict)


def tiny(n_ops=10_000):
    return Workload("tiny-1MiB", 1 * MiB, 256, lambda: TinyRandom(n_ops=n_ops),
                    "1 MiB arena, min block 256 B, 10,000 ops in batches of 64, 40% free")


def large(n_ops=10_000_000, batch=65_536, arena=16 * GiB):
    return Workload("large-16GiB", arena, 512, lambda: Lifetimes(n_ops=n_ops, batch=batch),
                    "16 GiB arena, min block 512 B, 10M ops in batches of 65,536, geometric lifetimes mean 1000 ops")


def frag(n_fill=1_000_000, n_big=50_000, batch=16_384, arena=4 * GiB):
    return Workload("frag-4GiB", arena, 256,
                    lambda: FragStress(n_fill=n_fill, n_big=n_big, batch=batch),
                    "4 GiB arena, min block 256 B, fill 1M x 4 KiB, free evens, 50k big, free all")


def usage(n_ops=5000, slots=64, batch=1, arena=4 * GiB):
    return Workload("usage-4GiB", arena, 4 * KiB, lambda: RandomSlots(n_ops=n_ops, slots=slots, batch=batch),
                    "4 GiB arena, min block 4 KiB, 5,000 ops on 64 slots (free if held, else malloc "
                    "log-uniform 1 kB-16 MB), one op per batch")


def objects(n_ops=200_000, batch=256, pool=1 * MiB):
    return Workload("objects-1MiB", pool, 8, lambda: TinyRandom(n_ops=n_ops, batch=batch, p_free=0.45, lo=8, hi=512),
                    "1 MiB pool of 8-byte units, 200,000 ops in batches of 256, 45% free, objects log-uniform "
                    "8-512 B")


def drain(client, alloc_batch):
    """Run a client to completion against ``alloc_batch(frees, sizes) -> out``.

    Returns the list of ``(frees, sizes, out)``."""
    trace = []
    while True:
        b = client.next_batch()
        if b is None:
            return trace
        out = alloc_batch(*b)
        client.feed(out)
        trace.append((b[0], b[1], np.asarray(out, np.uint64)))
