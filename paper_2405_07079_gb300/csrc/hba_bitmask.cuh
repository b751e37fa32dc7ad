// hba_bitmask.cuh -- the bitmask pool (§3.2) on the GPU.
//
// The pool is cut into units of min_block bytes.  One bit per unit says
// whether the unit is free (a set bit is free); a second bitmap marks the
// first unit of every in-use block, so that a free, which names only an
// address, knows where its block ends (the next marked or free unit).
// Allocation of k units (any k up to the pool) takes, by next fit, the
// lowest start at or after the rover where k consecutive units are free,
// else the lowest start of all; a run never wraps past the end of the pool.
//
// One CTA per pool.  Both bitmaps are copied into shared memory for the
// batch and written back at the end.  Frees are resolved NT at a time, in
// parallel: a free's validity and block end do not depend on the other
// frees of the batch (see the free phase below).  Allocations are applied
// one at a time in index order by warp 0, which holds the rover in
// registers and takes the rover itself when k units from it are free, else
// looks for the lowest start in the BM_QUICK words from the rover's word on,
// 32 words a step.  A request it does not settle there (or of more than 64
// units) goes to a CTA-wide scan:
//   k <= 64: thread t takes word w and computes the mask of starts in w that
//     have k free units, across w and w + 1 (128-bit AND of the shifted
//     words, built by doubling); the lowest start is an atomicMin, and the
//     scan stops after the first group of words holding one.
//   k > 64: a run this long leaves the word it starts in through its top
//     bit, so the lowest start in word w is where w's leading free bits begin
//     (or the rover, in the rover's word), and its length is those bits plus
//     the free units from word w + 1 on: 64 per full word up to the next
//     word that is not full, plus that word's trailing free bits.  Each
//     thread owns a contiguous segment of words; a block-wide suffix minimum
//     gives every segment the next non-full word after it.
// Within a batch's allocations free space only shrinks, so once k units
// cannot be found, every later request of k or more fails at once.
#pragma once

#include "hba_engine.cuh"

namespace hba {

constexpr uint32_t BM_MAX_WORDS = 12288;       // 786,432 units: both bitmaps in 192 KiB of shared memory

struct BmHdr {
    uint64_t wbase;  // first word of the pool's bitmaps in the word pools
    uint32_t words;  // ceil(units / 64)
    uint32_t rover;  // units
};

// Canonical state (the oracle's layout) from host copies of the bitmaps:
// pool bytes, unit, nblocks, (offset, size) per in-use block, rover (bytes).
inline size_t bm_export(const Arena& ar, const BmHdr& H, const uint64_t* F, const uint64_t* S, uint64_t* buf,
                        size_t cap) {
    size_t n = 0;
    auto put = [&](uint64_t v) { if (n < cap) buf[n] = v; ++n; };
    const uint32_t N = ar.G, lg = ar.lg;
    auto bit = [](const uint64_t* m, uint32_t u) { return (m[u >> 6] >> (u & 63)) & 1ull; };
    put((uint64_t)N << lg);
    put(1ull << lg);
    const size_t at = n;
    put(0);
    uint64_t cnt = 0;
    for (uint32_t p = 0; p < N; ++p) {
        if (!bit(S, p)) continue;
        uint32_t e = p + 1;
        while (e < N && !bit(F, e) && !bit(S, e)) ++e;
        put((uint64_t)p << lg);
        put((uint64_t)(e - p) << lg);
        ++cnt;
    }
    if (at < cap) buf[at] = cnt;
    put((uint64_t)H.rover << lg);
    return n;
}

#ifndef HBA_EMULATE
// (hi:lo) >> s for 0 <= s < 128, low word.
__device__ __forceinline__ uint64_t bm_shr_lo(uint64_t lo, uint64_t hi, uint32_t s) {
    if (s == 0) return lo;
    if (s >= 64) return hi >> (s - 64);
    return (lo >> s) | (hi << (64 - s));
}
__device__ __forceinline__ uint64_t bm_shr_hi(uint64_t hi, uint32_t s) {
    if (s >= 64) return 0;
    return hi >> s;
}

// Starts within word lo (bit b = unit 64 w + b) where k consecutive units,
// running into the next word hi, are all set.
__device__ __forceinline__ uint64_t bm_run_starts(uint64_t lo, uint64_t hi, uint32_t k) {
    uint64_t yl = ~0ull, pl = lo, ph = hi;
    uint32_t acc = 0;
    for (uint32_t i = 0; (1u << i) <= k; ++i) {
        const uint32_t len = 1u << i;
        if (k & len) {
            yl &= bm_shr_lo(pl, ph, acc);
            acc += len;
        }
        if ((2u << i) <= k) {  // P <- AND of 2 len shifts
            const uint64_t nl = pl & bm_shr_lo(pl, ph, len);
            const uint64_t nh = ph & bm_shr_hi(ph, len);
            pl = nl;
            ph = nh;
        }
    }
    return yl;
}

// Words from the rover's word that warp 0 searches before it hands a
// request to the whole CTA.
#ifndef HBA_BM_QUICK
#define HBA_BM_QUICK 256
#endif
constexpr uint32_t BM_QUICK = HBA_BM_QUICK;

constexpr uint32_t BM_HT = 512;  // hash slots of a chunk of frees (at least twice NT)

template <int NT>
struct BmSmem {
    static_assert(BM_HT >= 2 * NT && (BM_HT & (BM_HT - 1)) == 0, "free hash table");
    uint32_t rover, kfail, found, found_any, esc;
    uint32_t wmin[NT / 32];  // per-warp minima of the long-run search
    uint32_t hkey[BM_HT];    // frees of a chunk: start unit of each slot (NONE: empty)
    uint32_t hidx[BM_HT];    //   the lowest free index (in the chunk) naming it
    int64_t cnt[6];  // alloc_ok, alloc_fail, free_ok, free_fail, used units, requested bytes
    uint32_t err;
};

// Lowest start of k > 64 free units (whole CTA; F in shared memory, W
// words): at or after the rover if there is one, else the lowest of all;
// 0xFFFFFFFF if none.  Every thread returns the same value.
template <int NT>
__device__ uint32_t bm_long_search(BmSmem<NT>& S_, const uint64_t* F, uint32_t W, uint32_t rover, uint32_t k) {
    constexpr uint32_t NONE = 0xFFFFFFFFu;
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // segment of words [lo, hi) per thread; an odd length keeps the 16
    // threads of a half-warp on distinct 8-byte bank pairs
    const uint32_t c = ((W + NT - 1) / NT) | 1u;
    const uint32_t lo = min(t * c, W), hi = min(lo + c, W);
    uint32_t nf = W;  // first non-full word of the segment
    for (uint32_t x = lo; x < hi; ++x)
        if (F[x] != ~0ull) { nf = x; break; }
    // exclusive suffix minimum over threads: the first non-full word after the segment
    uint32_t v = nf;
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + o < 32) v = min(v, u);
    }
    uint32_t after = __shfl_down_sync(0xffffffffu, v, 1);
    if (lane == 31) after = W;
    if (lane == 0) S_.wmin[warp] = v;
    if (t == 0) {
        S_.found = NONE;
        S_.found_any = NONE;
    }
    __syncthreads();
    for (uint32_t q = warp + 1; q < NT / 32; ++q) after = min(after, S_.wmin[q]);
    const uint32_t w0 = rover >> 6, rb = rover & 63;
    uint32_t best0 = NONE, best1 = NONE;  // at or after the rover; anywhere
    uint32_t nz = after;                  // next non-full word after x
    for (uint32_t x = hi; x-- > lo;) {
        const uint64_t f = F[x];
        const uint32_t lead = (uint32_t)__clzll((long long)~f);  // free bits at the top of the word
        if (lead) {
            const uint32_t tail = 64u * (nz - x - 1) + (nz < W ? ctz64(~F[nz]) : 0u);  // free units from word x + 1
            const uint32_t b = 64u - lead;
            if (lead + tail >= k) best1 = (x << 6) + b;
            if (x > w0) {
                if (lead + tail >= k) best0 = (x << 6) + b;
            } else if (x == w0) {  // the rover's word: starts at or after the rover only
                const uint32_t bb = max(b, rb);
                if (64u - bb + tail >= k) best0 = (x << 6) + bb;
            }
        }
        if (f != ~0ull) nz = x;
    }
    if (best0 != NONE) atomicMin(&S_.found, best0);
    if (best1 != NONE) atomicMin(&S_.found_any, best1);
    __syncthreads();
    const uint32_t r = S_.found != NONE ? S_.found : S_.found_any;
    __syncthreads();
    return r;
}

// Allocation of k units at p (p + k <= N): clear F over [p, p + k), mark
// p, write the result (one thread; the caller moves the rover).
template <int NT>
__device__ void bm_take(BmSmem<NT>& S_, uint64_t* F, uint64_t* S, uint32_t lg, uint32_t p, uint32_t k, uint64_t sz,
                        uint64_t* res) {
    for (uint32_t q = p; q < p + k;) {
        const uint32_t qw = q >> 6, qb = q & 63;
        const uint32_t take = min(64u - qb, p + k - q);
        const uint64_t m = take == 64 ? ~0ull : ((1ull << take) - 1ull) << qb;
        F[qw] &= ~m;
        q += take;
    }
    S[p >> 6] |= 1ull << (p & 63);
    *res = (uint64_t)p << lg;
    ++S_.cnt[0];
    S_.cnt[4] += k;
    S_.cnt[5] += (int64_t)sz;
}

// The bitmaps of one pool in shared memory: F (free) and S (starts), W words each.
template <int NT>
__device__ void bm_pool(BmSmem<NT>& S_, Arena& ar, BmHdr& H, uint64_t* gF, uint64_t* gS, uint64_t* F, uint64_t* S,
                        const uint64_t* frees, uint8_t* fstat, uint32_t f0, uint32_t f1, const uint64_t* sizes,
                        uint64_t* out, uint32_t a0, uint32_t a1) {
    const uint32_t t = threadIdx.x;
    const uint32_t W = H.words, N = ar.G, lg = ar.lg;
    for (uint32_t w = t; w < W; w += NT) {
        F[w] = gF[w];
        S[w] = gS[w];
    }
    if (t == 0) {
        S_.rover = H.rover;
        S_.kfail = 0xFFFFFFFFu;
        for (int q = 0; q < 6; ++q) S_.cnt[q] = 0;
        S_.err = 0;
    }
    __syncthreads();
    // ---- frees, NT at a time.  A free is valid when it names a unit
    // boundary inside the pool whose start bit is set; its block ends at the
    // next free or marked unit.  No other free of the batch moves that end
    // (a free only turns a marked start into free units), so the frees of a
    // chunk are resolved together: validity and ends first, then the bit
    // updates.  Of several frees of one block the lowest index applies and
    // the others are rejected, as they are one by one (the start bit is gone
    // by their turn); a later chunk finds the bit gone.
    constexpr uint32_t NONE = 0xFFFFFFFFu;
    for (uint32_t j0 = f0; j0 < f1; j0 += NT) {
        const uint32_t j = j0 + t;
        uint32_t p = NONE;
        if (j < f1) {
            const uint64_t off = frees[j];
            if ((off & ((1ull << lg) - 1)) == 0 && (off >> lg) < N) {
                const uint32_t q = (uint32_t)(off >> lg);
                if ((S[q >> 6] >> (q & 63)) & 1ull) p = q;
            }
        }
        for (uint32_t h = t; h < BM_HT; h += NT) {
            S_.hkey[h] = NONE;
            S_.hidx[h] = NONE;
        }
        __syncthreads();
        uint32_t slot = 0;
        if (p != NONE) {  // at most NT keys in BM_HT >= 2 NT slots: a free slot is always found
            slot = (p * 2654435761u) & (BM_HT - 1);
            for (uint32_t probe = 0; probe < BM_HT; ++probe) {
                const uint32_t key = atomicCAS(&S_.hkey[slot], NONE, p);
                if (key == NONE || key == p) break;
                slot = (slot + 1) & (BM_HT - 1);
            }
            atomicMin(&S_.hidx[slot], t);
        }
        __syncthreads();
        const bool ok = p != NONE && S_.hidx[slot] == t;
        uint32_t e = 0;
        if (ok) {
            const uint32_t pw = p >> 6, pb = p & 63;
            const uint64_t above = pb == 63 ? 0ull : ~0ull << (pb + 1);
            const uint64_t stop = (F[pw] | S[pw]) & above;
            if (stop) {
                e = (pw << 6) + ctz64(stop);
            } else {
                uint32_t x = pw + 1;
                while (x < W && (F[x] | S[x]) == 0ull) ++x;
                e = x < W ? (x << 6) + ctz64(F[x] | S[x]) : N;
            }
            if (e > N) e = N;
        }
        __syncthreads();  // every end is known before any bit changes
        if (ok) {
            for (uint32_t q = p; q < e;) {  // set F over [p, e), a word piece at a time
                const uint32_t qw = q >> 6, qb = q & 63;
                const uint32_t take = min(64u - qb, e - q);
                const uint64_t m = take == 64 ? ~0ull : ((1ull << take) - 1ull) << qb;
                atomicOr(reinterpret_cast<unsigned long long*>(&F[qw]), (unsigned long long)m);
                q += take;
            }
            atomicAnd(reinterpret_cast<unsigned long long*>(&S[p >> 6]), ~(1ull << (p & 63)));
        }
        if (j < f1 && fstat) fstat[j] = ok ? 0 : 1;
        const uint32_t n_ok = __popc(__ballot_sync(0xffffffffu, ok));
        const uint32_t n_bad = __popc(__ballot_sync(0xffffffffu, j < f1 && !ok));
        const uint32_t units = __reduce_add_sync(0xffffffffu, ok ? e - p : 0u);
        if ((t & 31) == 0) {
            if (n_ok) atomicAdd(reinterpret_cast<unsigned long long*>(&S_.cnt[2]), (unsigned long long)n_ok);
            if (n_bad) atomicAdd(reinterpret_cast<unsigned long long*>(&S_.cnt[3]), (unsigned long long)n_bad);
            if (units) atomicAdd(reinterpret_cast<unsigned long long*>(&S_.cnt[4]), (unsigned long long)(-(int64_t)units));
        }
        __syncthreads();
    }
    // ---- allocations in index order.  Warp 0 applies them one by one and
    // looks for each run in the BM_QUICK words from the rover's word on
    // (32 words a step, no block barrier); that finds the lowest start at or
    // after the rover whenever there is one in those words.  A request it
    // does not settle (no start there, or more than 64 units) is searched by
    // the whole CTA, after which warp 0 goes on.
    const uint64_t P = (uint64_t)N << lg;
    uint32_t i = a0;
    while (true) {
        if (t < 32) {
            uint32_t rover = S_.rover, kfail = S_.kfail;  // warp-uniform; stored back below
            uint32_t esc = a1;
            for (uint32_t j0 = i; j0 < a1 && esc == a1; j0 += 32) {
                const uint64_t mine = j0 + t < a1 ? sizes[j0 + t] : 0ull;
                const uint32_t nq = a1 - j0 < 32u ? a1 - j0 : 32u;
                for (uint32_t q = 0; q < nq; ++q) {
                    const uint64_t sz = __shfl_sync(0xffffffffu, mine, q);  // every lane, every step
                    const uint32_t k = (sz == 0 || sz > P) ? 0u : (uint32_t)((sz + (1ull << lg) - 1) >> lg);
                    if (k == 0 || k > N || k >= kfail) {
                        if (t == 0) {
                            out[j0 + q] = FAIL64;
                            ++S_.cnt[1];
                        }
                        continue;
                    }
                    if (k > 64) {
                        esc = j0 + q;
                        break;
                    }
                    uint32_t p = NONE;
                    if (rover + k <= N) {  // the rover itself, when k units from it are free
                        const uint32_t w = rover >> 6, b = rover & 63;
                        uint64_t v = F[w] >> b;
                        if (b && w + 1 < W) v |= F[w + 1] << (64 - b);
                        const uint64_t m = k == 64 ? ~0ull : (1ull << k) - 1ull;
                        if ((v & m) == m) p = rover;
                    }
                    const uint32_t w0 = rover >> 6;
                    const uint32_t wend = p != NONE ? w0 : (W - w0 < BM_QUICK ? W : w0 + BM_QUICK);
                    for (uint32_t c0 = w0; c0 < wend; c0 += 32) {
                        const uint32_t w = c0 + t;
                        uint64_t v = 0;
                        if (w < wend) {
                            v = bm_run_starts(F[w], w + 1 < W ? F[w + 1] : 0ull, k);
                            if (w == w0) v &= (rover & 63) ? ~0ull << (rover & 63) : ~0ull;
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, v != 0);
                        if (bal) {
                            const int src = __ffs((int)bal) - 1;
                            const uint64_t vv = __shfl_sync(0xffffffffu, v, src);
                            p = ((c0 + (uint32_t)src) << 6) + ctz64(vv);
                            break;
                        }
                    }
                    if (p == NONE) {
                        esc = j0 + q;
                        break;
                    }
                    if (p + k > N) {  // the lowest start runs off the end: nothing of k units is free
                        if (t == 0) {
                            out[j0 + q] = FAIL64;
                            ++S_.cnt[1];
                        }
                        kfail = k;
                        continue;
                    }
                    if (t == 0) bm_take(S_, F, S, lg, p, k, sz, out + j0 + q);
                    rover = p + k;
                    __syncwarp();
                }
            }
            if (t == 0) {
                S_.esc = esc;
                S_.rover = rover;
                S_.kfail = kfail;
            }
        }
        __syncthreads();
        const uint32_t e = S_.esc;
        if (e >= a1) break;
        // request e by the whole CTA: pass 0, starts >= rover in words
        // [w0, W); pass 1, words [0, min(w0 + 1, W)); runs of more than 64
        // units by the segment search
        const uint64_t sz = sizes[e];
        const uint32_t k = (uint32_t)((sz + (1ull << lg) - 1) >> lg);
        const uint32_t rover = S_.rover;
        if (k > 64) {
            const uint32_t p = bm_long_search<NT>(S_, F, W, rover, k);
            if (t == 0) S_.found = p;
            __syncthreads();
        } else {
            const uint32_t w0 = rover >> 6 < W ? rover >> 6 : W;
            if (t == 0) S_.found = 0xFFFFFFFFu;
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass) {
                const uint32_t wlo = pass == 0 ? w0 : 0u;
                const uint32_t whi = pass == 0 ? W : (w0 + 1 < W ? w0 + 1 : W);
                for (uint32_t c0 = wlo; c0 < whi; c0 += NT) {
                    const uint32_t w = c0 + t;
                    if (w < whi) {
                        uint64_t v = bm_run_starts(F[w], w + 1 < W ? F[w + 1] : 0ull, k);
                        if (pass == 0 && w == w0) v &= (rover & 63) ? ~0ull << (rover & 63) : ~0ull;
                        if (v) atomicMin(&S_.found, (w << 6) + ctz64(v));
                    }
                    __syncthreads();
                    const bool got = S_.found != 0xFFFFFFFFu;
                    __syncthreads();
                    if (got) break;
                }
                if (S_.found != 0xFFFFFFFFu) break;
            }
        }
        if (t == 0) {
            const uint32_t p = S_.found;
            if (p == NONE || p + k > N) {
                out[e] = FAIL64;
                ++S_.cnt[1];
                S_.kfail = k;
            } else {
                bm_take(S_, F, S, lg, p, k, sz, out + e);
                S_.rover = p + k;
            }
        }
        i = e + 1;
        __syncthreads();
    }
    for (uint32_t w = t; w < W; w += NT) {
        gF[w] = F[w];
        gS[w] = S[w];
    }
    if (t == 0) {
        H.rover = S_.rover;
        ar.alloc_ok += S_.cnt[0];
        ar.alloc_fail += S_.cnt[1];
        ar.free_ok += S_.cnt[2];
        ar.free_fail += S_.cnt[3];
        ar.used_g += S_.cnt[4];
        ar.used_blocks += S_.cnt[0] - S_.cnt[2];
        ar.requested += S_.cnt[5];
    }
    __syncthreads();
}
#endif

}  // namespace hba
