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
// batch and written back at the end.  Frees are applied one at a time by
// lane 0 of warp 0 (the warp loads 32 offsets at a time), a few word
// operations each.  An allocation is a CTA-wide scan:
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

template <int NT>
struct BmSmem {
    uint64_t sz[NT];  // the current group of request sizes
    uint32_t rover, kfail, found, found_any;
    uint32_t wmin[NT / 32];  // per-warp minima of the long-run search
    int64_t cnt[6];  // alloc_ok, alloc_fail, free_ok, free_fail, used units, requested bytes
    uint32_t err;
};

// Free the block that starts at byte offset off (one thread).
template <int NT>
__device__ void bm_free_one(BmSmem<NT>& S_, uint64_t* F, uint64_t* S, uint32_t W, uint32_t N, uint32_t lg,
                            uint64_t off, uint8_t* fstat, uint32_t j) {
    uint32_t st = 1;
    if ((off & ((1ull << lg) - 1)) == 0 && (off >> lg) < N) {
        const uint32_t p = (uint32_t)(off >> lg);
        const uint32_t pw = p >> 6, pb = p & 63;
        if ((S[pw] >> pb) & 1ull) {
            // the block ends at the next free or marked unit, or the pool's end
            const uint64_t above = pb == 63 ? 0ull : ~0ull << (pb + 1);
            const uint64_t stop = (F[pw] | S[pw]) & above;
            uint32_t e;
            if (stop) {
                e = (pw << 6) + ctz64(stop);
            } else {
                uint32_t x = pw + 1;
                while (x < W && (F[x] | S[x]) == 0ull) ++x;
                e = x < W ? (x << 6) + ctz64(F[x] | S[x]) : N;
            }
            if (e > N) e = N;
            for (uint32_t q = p; q < e;) {  // set F over [p, e), a word piece at a time
                const uint32_t qw = q >> 6, qb = q & 63;
                const uint32_t take = min(64u - qb, e - q);
                const uint64_t m = take == 64 ? ~0ull : ((1ull << take) - 1ull) << qb;
                F[qw] |= m;
                q += take;
            }
            S[pw] &= ~(1ull << pb);
            S_.cnt[4] -= (int64_t)(e - p);
            st = 0;
        }
    }
    if (fstat) fstat[j] = (uint8_t)st;
    ++S_.cnt[st ? 3 : 2];
}

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
    // ---- frees, one by one (lane 0 of warp 0; the warp loads 32 offsets at a time)
    if (t < 32) {
        for (uint32_t j0 = f0; j0 < f1; j0 += 32) {
            const uint64_t mine = j0 + t < f1 ? frees[j0 + t] : 0ull;
            const uint32_t nq = f1 - j0 < 32u ? f1 - j0 : 32u;
            for (uint32_t q = 0; q < nq; ++q) {
                const uint64_t off = __shfl_sync(0xffffffffu, mine, q);  // every lane, every step
                if (t == 0) bm_free_one(S_, F, S, W, N, lg, off, fstat, j0 + q);
                __syncwarp();
            }
        }
    }
    __syncthreads();
    // ---- allocations, one by one, each a CTA-wide run search
    const uint64_t P = (uint64_t)N << lg;
    for (uint32_t i = a0; i < a1; ++i) {
        if ((i - a0) % NT == 0) {  // the next NT sizes, loaded together
            __syncthreads();
            if (i + t < a1) S_.sz[t] = sizes[i + t];
            __syncthreads();
        }
        const uint64_t sz = S_.sz[(i - a0) % NT];
        const uint32_t k = (sz == 0 || sz > P) ? 0u : (uint32_t)((sz + (1ull << lg) - 1) >> lg);
        if (k == 0 || k > N || k >= S_.kfail) {  // uniform: S_.kfail changes behind barriers
            if (t == 0) {
                out[i] = FAIL64;
                ++S_.cnt[1];
            }
            continue;
        }
        const uint32_t rover = S_.rover;
        if (k > 64) {
            const uint32_t p = bm_long_search<NT>(S_, F, W, rover, k);
            if (t == 0) S_.found = p;
            __syncthreads();
        } else {
        const uint32_t w0 = rover >> 6 < W ? rover >> 6 : W;
        if (t == 0) S_.found = 0xFFFFFFFFu;
        __syncthreads();
        // pass 0: starts >= rover in words [w0, W); pass 1: words [0, min(w0 + 1, W))
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
            if (p == 0xFFFFFFFFu || p + k > N) {
                out[i] = FAIL64;
                ++S_.cnt[1];
                S_.kfail = k;
            } else {
                for (uint32_t q = p; q < p + k;) {  // clear F over [p, p + k)
                    const uint32_t qw = q >> 6, qb = q & 63;
                    const uint32_t take = min(64u - qb, p + k - q);
                    const uint64_t m = take == 64 ? ~0ull : ((1ull << take) - 1ull) << qb;
                    F[qw] &= ~m;
                    q += take;
                }
                S[p >> 6] |= 1ull << (p & 63);
                S_.rover = p + k;
                out[i] = (uint64_t)p << lg;
                ++S_.cnt[0];
                S_.cnt[4] += k;
                S_.cnt[5] += (int64_t)sz;
            }
        }
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
