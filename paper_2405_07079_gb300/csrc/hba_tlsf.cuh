// hba_tlsf.cuh -- two-level segregated fit (§5.2) on the GPU.
//
// §5.2 keeps Algorithms 4 and 5 and changes only the lookup: a first-level
// bitmap over the power-of-two classes, each of whose bits says that a
// second-level bitmap is non-zero; the second level splits a class linearly
// into lists, and a set bit there says that list is non-empty.
//
// Sizes here are in granules (min_block units).  With 16 lists per class
// (the paper gives no count), the list of a free block of r granules is
// (f, s): f = floor(log2 r) and s the four bits below the leading one, so
// list (f, s) holds the sizes [2^f + s 2^f / 16, 2^f + (s + 1) 2^f / 16).
// In bytes the same block is in list (f + log2 min_block, s): the lists are
// the byte lists shifted, which is how they are exported.
//
// An allocation of r granules takes the lowest non-empty list whose lower
// bound is >= r, so that every block of that list fits -- the two-level
// analogue of the strict class rule of §5.1.  That list is found by rounding
// r up to the next list bound and searching the second-level bitmap of its
// class, then the first-level bitmap above it.
//
// Records are the segregated-fit engine's (x = size | state, y = prev_adj,
// z = next in list, w = previous in list), so the arena header's counters,
// the extent scan and the canonical export of the blocks carry over; the
// list heads and bitmaps live in a TlsfLists per arena.
//
// Execution: the batch engine (hba_engine.cuh, class layout POL 1) applies
// TLSF batches on the GPU, as it does segregated-fit ones.  This file keeps
// the list operations one at a time: the serial batch below is the host
// emulation's second implementation of the policy, and the export and
// initial state serve every TLSF handle.
#pragma once

#include "hba_engine.cuh"

namespace hba {

// The list constants, TlsfLists, tl_list and tl_bound are in hba_engine.cuh
// (the batch engine runs this policy too).

// Lowest non-empty list at or above list t, or TL_NONE.
HBA_HD uint32_t tl_find(const TlsfLists& L, uint32_t t) {
    const uint32_t f = t / TL_SL, s = t % TL_SL;
    const uint32_t here = (uint32_t)L.slmask[f] & (0xFFFFu << s) & 0xFFFFu;
    if (here) return f * TL_SL + ctz64(here);
    const uint32_t up = f + 1 < TL_FL ? (L.flmask >> (f + 1)) << (f + 1) : 0u;
    if (!up) return TL_NONE;
    const uint32_t f2 = ctz64(up);
    return f2 * TL_SL + ctz64(L.slmask[f2]);
}

HBA_HD void tl_mark(TlsfLists& L, uint32_t list, bool nonempty) {
    const uint32_t f = list / TL_SL, s = list % TL_SL;
    if (nonempty) L.slmask[f] = (uint16_t)(L.slmask[f] | (1u << s));
    else L.slmask[f] = (uint16_t)(L.slmask[f] & ~(1u << s));
    if (L.slmask[f]) L.flmask |= 1u << f;
    else L.flmask &= ~(1u << f);
}

// Push block [g, g + r) with prev_adj pa at the head of its list.
HBA_HD void tl_push(TlsfLists& L, Rec* rec, uint32_t g, uint32_t r, uint32_t pa) {
    const uint32_t k = tl_list(r);
    const uint32_t head = L.heads[k];
    rec[g] = Rec{mkx(r, ST_FREE), pa, head, NIL};
    if (head != NIL) rec[head].w = g;
    L.heads[k] = g;
    tl_mark(L, k, true);
}

// Unlink a free block (its record rg) from its list.
HBA_HD void tl_unlink(TlsfLists& L, Rec* rec, const Rec& rg) {
    const uint32_t k = tl_list(sz_of(rg.x));
    if (rg.w != NIL) rec[rg.w].z = rg.z;
    else L.heads[k] = rg.z;
    if (rg.z != NIL) rec[rg.z].w = rg.w;
    if (L.heads[k] == NIL) tl_mark(L, k, false);
}

// Counters of one batch, added to the arena header at the end.
struct TlCount {
    int64_t aok = 0, afail = 0, fok = 0, ffail = 0, usedg = 0, blocks = 0, req = 0;
};

// Algorithm 5 for the block at byte offset `off` (§5.2 lookup).  Returns 0
// when applied, 1 when rejected (not the start of an in-use block).
HBA_HD uint32_t tl_free_one(TlsfLists& L, Rec* rec, uint64_t A, uint32_t G, uint32_t lg, uint64_t off,
                            TlCount& c) {
    if (off >= A || (off & ((1ull << lg) - 1)) != 0) {
        ++c.ffail;
        return 1;
    }
    const uint32_t g = (uint32_t)(off >> lg);
    const Rec r = rec[g];
    if (st_of(r.x) != ST_USED) {
        ++c.ffail;
        return 1;
    }
    const uint32_t sz = sz_of(r.x);
    uint32_t start = g, size = sz, pa = r.y;
    if (r.y != NIL) {
        const Rec rl = rec[r.y];
        if (st_of(rl.x) == ST_FREE) {  // coalesce with the left block
            tl_unlink(L, rec, rl);
            start = r.y;
            size += sz_of(rl.x);
            pa = rl.y;
            rec[g].x = 0;
            --c.blocks;
        }
    }
    const uint32_t right = g + sz;
    if (right < G) {
        const Rec rr = rec[right];
        if (st_of(rr.x) == ST_FREE) {  // coalesce with the right block
            tl_unlink(L, rec, rr);
            size += sz_of(rr.x);
            rec[right].x = 0;
            --c.blocks;
        }
    }
    if (start + size < G) rec[start + size].y = start;
    tl_push(L, rec, start, size, pa);
    ++c.fok;
    c.usedg -= sz;
    return 0;
}

// Request size in granules, or 0 when it cannot be served at all (size 0 or
// above the arena).
HBA_HD uint32_t tl_granules(uint64_t s, uint64_t A, uint32_t lg) {
    if (s == 0 || s > A) return 0;
    return (uint32_t)((s + (1ull << lg) - 1) >> lg);
}

// Algorithm 4 for r granules from list k (non-empty, lower bound >= r).
// Returns the block's granule; counts the allocation.
HBA_HD uint32_t tl_take(TlsfLists& L, Rec* rec, uint32_t G, uint32_t k, uint32_t r, TlCount& c) {
    const uint32_t Y = L.heads[k];
    const Rec ry = rec[Y];
    L.heads[k] = ry.z;
    if (ry.z != NIL) {
#ifdef __CUDA_ARCH__
        prefetch_l2(rec + ry.z);  // the new head: the next pop of this list reads it
#endif
        rec[ry.z].w = NIL;
    } else {
        tl_mark(L, k, false);
    }
    const uint32_t ysz = sz_of(ry.x);
    rec[Y] = Rec{mkx(r, ST_USED), ry.y, NIL, NIL};
    if (ysz > r) {  // split: the remainder goes to the head of its list
        tl_push(L, rec, Y + r, ysz - r, Y);
        if (Y + ysz < G) rec[Y + ysz].y = Y + r;
        ++c.blocks;
    }
    ++c.aok;
    c.usedg += r;
    return Y;
}

// Whole batch, one op at a time (the host emulation).
HBA_HD void tl_batch_serial(TlsfLists& L, Rec* rec, uint64_t A, uint32_t G, uint32_t lg, const uint64_t* frees,
                            uint32_t nf, uint8_t* fstat, const uint64_t* sizes, uint32_t na, uint64_t* out,
                            TlCount& c) {
    for (uint32_t j = 0; j < nf; ++j) {
        const uint32_t st = tl_free_one(L, rec, A, G, lg, frees[j], c);
        if (fstat) fstat[j] = (uint8_t)st;
    }
    for (uint32_t i = 0; i < na; ++i) {
        const uint32_t r = tl_granules(sizes[i], A, lg);
        const uint32_t k = r && r <= G ? tl_find(L, tl_bound(r)) : TL_NONE;
        if (k == TL_NONE) {
            out[i] = FAIL64;
            ++c.afail;
            continue;
        }
        out[i] = (uint64_t)tl_take(L, rec, G, k, r, c) << lg;
        c.req += (int64_t)sizes[i];
    }
}

HBA_HD void tl_apply_counts(Arena& ar, const TlsfLists& L, const TlCount& c) {
    ar.mask = L.flmask;
    ar.alloc_ok += c.aok;
    ar.alloc_fail += c.afail;
    ar.free_ok += c.fok;
    ar.free_fail += c.ffail;
    ar.used_g += c.usedg;
    ar.used_blocks += c.aok - c.fok;
    ar.blocks += c.blocks;
    ar.requested += c.req;
}

// Initial lists of an arena of G granules: one free block [0, G).
inline void tl_init_host(TlsfLists* L, uint32_t G) {
    memset(L, 0, sizeof(*L));
    for (uint32_t k = 0; k < TL_NL; ++k) L->heads[k] = NIL;
    const uint32_t k = tl_list(G);
    L->heads[k] = 0;
    tl_mark(*L, k, true);
}

// Canonical state of a TLSF arena (the oracle's layout): blocks in address
// order, the 64 x 16 byte lists head to tail, the first-level bitmap over
// byte classes, the 64 second-level bitmaps.
inline size_t tl_export(const Arena& ar, const TlsfLists& L, const Rec* rec, uint64_t* buf, size_t cap) {
    size_t n = 0;
    auto put = [&](uint64_t v) { if (n < cap) buf[n] = v; ++n; };
    const uint64_t mb = 1ull << ar.lg;
    put(ar.arena_bytes);
    put(mb);
    put((uint64_t)ar.blocks);
    uint32_t g = 0;
    uint64_t guard = 0;
    while (g < ar.G) {
        const Rec r = rec[g];
        const uint32_t sz = sz_of(r.x), st = st_of(r.x);
        if (sz == 0 || (st != ST_USED && st != ST_FREE) || ++guard > ar.G) { put(~0ull); break; }
        put((uint64_t)g * mb);
        put((uint64_t)sz * mb | ((uint64_t)(st == ST_FREE) << 63));
        g += sz;
    }
    for (uint32_t kb = 0; kb < 64 * TL_SL; ++kb) {
        const int f = (int)(kb / TL_SL) - (int)ar.lg;
        const size_t at = n;
        put(0);
        uint64_t cnt = 0;
        if (f >= 0 && f < (int)TL_FL) {
            for (uint32_t h = L.heads[(uint32_t)f * TL_SL + kb % TL_SL]; h != NIL && cnt <= ar.G; ++cnt) {
                put((uint64_t)h * mb);
                h = rec[h].z;
            }
        }
        if (at < cap) buf[at] = cnt;
    }
    put((uint64_t)L.flmask << ar.lg);
    for (int fb = 0; fb < 64; ++fb) {
        const int f = fb - (int)ar.lg;
        put(f >= 0 && f < (int)TL_FL ? (uint64_t)L.slmask[f] : 0ull);
    }
    return n;
}


}  // namespace hba
