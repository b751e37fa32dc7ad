"""Shared test helpers: drive a workload through the oracle and a device path."""
from __future__ import annotations

import numpy as np

FAIL = np.uint64(0xFFFFFFFFFFFFFFFF)


def oracle_trace(wl, max_batches=None, policy="segfit"):
    """Run the workload's client closed-loop against the oracle.

    Returns (trace, oracle) where trace is a list of
    (frees, sizes, out, status) with the oracle's results."""
    import oracle

    o = oracle.Oracle(wl.arena, wl.min_block, policy)
    cl = wl.make()
    trace = []
    while max_batches is None or len(trace) < max_batches:
        b = cl.next_batch()
        if b is None:
            break
        f, s = b
        out, st = o.batch(f, s)
        cl.feed(out)
        trace.append((f, s, out, st))
    return trace, o


def to_dev(a: np.ndarray, dev):
    import torch

    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def from_dev(t) -> np.ndarray:
    import torch

    a = t.cpu().numpy()
    return a.view(np.uint64) if t.dtype == torch.int64 else a


def first_diff(a, b):
    d = np.nonzero(np.asarray(a) != np.asarray(b))[0]
    return int(d[0]) if d.size else None


def check_invariants(words):
    """Invariants of a canonical state (T2): blocks tile the arena, no two
    adjacent free blocks, every free block in exactly one list and in the list
    of floor(log2 size), the bitmap matches the non-empty lists, offsets and
    sizes are multiples of min_block."""
    from oracle import decode_state

    s = decode_state(words)
    A, mb = s["arena"], s["min_block"]
    pos = 0
    prev_free = False
    free_blocks = set()
    for off, sz, fr in s["blocks"]:
        assert off == pos and sz > 0 and off % mb == 0 and sz % mb == 0
        assert not (fr and prev_free), "two adjacent free blocks"
        prev_free = fr
        if fr:
            free_blocks.add((off, sz))
        pos = off + sz
    assert pos == A
    assert s["nblocks"] == len(s["blocks"])
    size_of = {o: z for o, z in free_blocks}
    listed = []
    mask = 0
    for k, lst in enumerate(s["bins"]):
        for o in lst:
            assert o in size_of and size_of[o].bit_length() - 1 == k, "block in the wrong list"
        listed += lst
        if lst:
            mask |= 1 << k
    assert sorted(listed) == sorted(size_of), "free blocks and list members differ"
    assert mask == s["bitmask"]
    return s


def canary_intact(guard, byte=0xA5, chunk=1 << 30) -> bool:
    """True iff every byte of the device tensor ``guard`` (uint8) still holds
    ``byte``: compared as 64-bit words, a chunk at a time, so that a guard of
    tens of GiB needs no guard-sized temporary."""
    import torch

    word = int.from_bytes(bytes([byte]) * 8, "little", signed=True)
    n = guard.numel()
    head = n - n % 8
    w = guard[:head].view(torch.int64)
    for i in range(0, w.numel(), chunk // 8):
        if not bool((w[i:i + chunk // 8] == word).all()):
            return False
    return bool((guard[head:] == byte).all()) if head < n else True
