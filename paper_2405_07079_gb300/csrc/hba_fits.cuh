// hba_fits.cuh -- the sequential fits on address-sorted lists (§3.1
// Algorithms 1 and 2, §4 Algorithm 3 and its first-fit and next-fit
// variants) on the GPU.
//
// State of an arena (sizes and addresses in granules):
//   - the free blocks, an array sorted by address (§3.1's free HAL);
//   - the in-use blocks, an array sorted by address (the used HAL);
//   - the next-fit rover (the end of the last allocated block).
// The HAL of §3.1 chunks these arrays so that a CPU shifts at most one chunk
// on an insert or a remove; here a CTA shifts a whole array, NT entries per
// step, which is the same result.
//
// One CTA per arena applies the batch one request at a time: frees in index
// order, then allocations.  Every request is CTA-wide work:
//   - positions in a sorted array come from a k-ary search: each round, every
//     thread tests one pivot and __syncthreads_count narrows the range NT-fold;
//   - an insert or a remove shifts the array tail by one, NT entries per step
//     (all loads of a step before any of its stores);
//   - the fit's candidate is a min-reduction over the free array: the lowest
//     index that fits (first fit; next fit from the rover's block, wrapping),
//     or the smallest size with the lowest index (best fit), stopping after
//     the step where an exact or first fit is found;
//   - allocations are classified NT at a time against the largest free
//     block: a request above it fails and changes nothing, so the requests
//     before the first that can be served are resolved at once.
// Control flow is uniform across the CTA: thread 0 writes the values every
// thread needs into shared memory before a barrier.
#pragma once

#include "hba_engine.cuh"

namespace hba {

constexpr uint32_t FIT_FIRST = 0, FIT_NEXT = 1, FIT_BEST = 2;

struct FitBlk {
    uint32_t a, z;  // first granule, granules
};

struct FitHdr {
    uint32_t nfree, nused, rover, fit;
};

// Canonical state of a sequential-fit arena (the oracle's layout): arena,
// min_block, nfree, (address, size) per free block, nused, (address, size)
// per used block, rover (bytes).
inline size_t fit_export(const Arena& ar, const FitHdr& H, const FitBlk* fa, const FitBlk* ua, uint64_t* buf,
                         size_t cap) {
    size_t n = 0;
    auto put = [&](uint64_t v) { if (n < cap) buf[n] = v; ++n; };
    const uint32_t lg = ar.lg;
    put(ar.arena_bytes);
    put(1ull << lg);
    put(H.nfree);
    for (uint32_t i = 0; i < H.nfree; ++i) { put((uint64_t)fa[i].a << lg); put((uint64_t)fa[i].z << lg); }
    put(H.nused);
    for (uint32_t i = 0; i < H.nused; ++i) { put((uint64_t)ua[i].a << lg); put((uint64_t)ua[i].z << lg); }
    put((uint64_t)H.rover << lg);
    return n;
}

#ifndef HBA_EMULATE
// Free and used arrays are worked on in shared memory while each holds at
// most FIT_RES entries; an insert that would pass that moves both to global
// memory for the rest of the batch.
#ifndef HBA_FIT_RES
#define HBA_FIT_RES 4096u
#endif
constexpr uint32_t FIT_RES = HBA_FIT_RES;

template <int NT>
struct FitSmem {
    uint64_t wz[NT];        // the current group of request sizes
    uint32_t nf, nu, rover, cap;
    uint32_t maxz;          // largest free block (valid when !dirty)
    uint32_t dirty;
    uint32_t v[8];          // broadcast slots
    unsigned long long best;
    int64_t cnt[6];         // alloc_ok, alloc_fail, free_ok, free_fail, used granules, requested bytes
    uint32_t err;
};

// Entries of arr[0, n) whose key (address, or end when by_end) is <= k.
template <int NT>
__device__ uint32_t fit_count_le(const FitBlk* arr, uint32_t n, uint32_t k, bool by_end) {
    const uint32_t t = threadIdx.x;
    uint32_t lo = 0, hi = n;  // the answer is in [lo, hi]
    while (hi - lo > (uint32_t)NT) {
        const uint32_t step = (hi - lo + NT - 1) / NT;
        const uint32_t idx = lo + t * step;
        bool le = false;
        if (idx < hi) {
            const FitBlk b = arr[idx];
            le = (by_end ? b.a + b.z : b.a) <= k;
        }
        const uint32_t c = (uint32_t)__syncthreads_count(le);
        if (c == 0) return lo;  // arr[lo] is already above k
        const uint32_t last = lo + (c - 1) * step;  // the last pivot at or below k
        const uint32_t nxt = lo + c * step;
        lo = last + 1;
        hi = nxt < hi ? nxt : hi;
    }
    bool le = false;
    if (lo + t < hi) {
        const FitBlk b = arr[lo + t];
        le = (by_end ? b.a + b.z : b.a) <= k;
    }
    return lo + (uint32_t)__syncthreads_count(le);
}

// Insert v at position p of arr[0, n) (n < capacity): the tail moves up by one.
template <int NT>
__device__ void fit_insert(FitBlk* arr, uint32_t n, uint32_t p, FitBlk v) {
    const uint32_t t = threadIdx.x;
    for (uint32_t top = n; top > p;) {  // entries [base, top) move to [base + 1, top + 1)
        const uint32_t base = top - p > (uint32_t)NT ? top - NT : p;
        FitBlk x{0, 0};
        const bool mine = base + t < top;
        if (mine) x = arr[base + t];
        __syncthreads();
        if (mine) arr[base + t + 1] = x;
        __syncthreads();
        top = base;
    }
    if (t == 0) arr[p] = v;
    __syncthreads();
}

// Remove position p of arr[0, n): the tail moves down by one.
template <int NT>
__device__ void fit_remove(FitBlk* arr, uint32_t n, uint32_t p) {
    const uint32_t t = threadIdx.x;
    for (uint32_t base = p + 1; base < n; base += NT) {  // [base, base + NT) moves to [base - 1, ...)
        FitBlk x{0, 0};
        const bool mine = base + t < n;
        if (mine) x = arr[base + t];
        __syncthreads();
        if (mine) arr[base + t - 1] = x;
        __syncthreads();
    }
}

// Largest free block (CTA-wide).
template <int NT>
__device__ void fit_refresh_max(FitSmem<NT>& S, const FitBlk* fa) {
    const uint32_t t = threadIdx.x;
    if (t == 0) S.v[7] = 0;
    __syncthreads();
    uint32_t m = 0;
    for (uint32_t i = t; i < S.nf; i += NT) m = max(m, fa[i].z);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) atomicMax(&S.v[7], m);
    __syncthreads();
    if (t == 0) {
        S.maxz = S.v[7];
        S.dirty = 0;
    }
    __syncthreads();
}

// The fit's candidate for s granules (some free block is >= s): its index.
template <int NT>
__device__ uint32_t fit_pick(FitSmem<NT>& S, const FitBlk* fa, uint32_t s, uint32_t fit) {
    const uint32_t t = threadIdx.x;
    const uint32_t nf = S.nf;
    uint32_t start = 0;
    if (fit == FIT_NEXT) start = fit_count_le<NT>(fa, nf, S.rover, true);  // first block ending above the rover
    if (t == 0) S.best = ~0ull;
    __syncthreads();
    for (uint32_t k0 = 0; k0 < nf; k0 += NT) {
        const uint32_t k = k0 + t;
        if (k < nf) {
            const uint32_t i = fit == FIT_NEXT ? (start + k < nf ? start + k : start + k - nf) : k;
            const FitBlk b = fa[i];
            if (b.z >= s) {
                // first / next fit: order of visit; best fit: (size, address order)
                const unsigned long long key = fit == FIT_BEST ? ((unsigned long long)b.z << 32) | i
                                                               : ((unsigned long long)k << 32) | i;
                atomicMin(&S.best, key);
            }
        }
        __syncthreads();
        const unsigned long long b = S.best;
        const bool done = b != ~0ull && (fit != FIT_BEST || (uint32_t)(b >> 32) == s);
        __syncthreads();
        if (done) break;
    }
    return (uint32_t)(S.best & 0xffffffffu);
}

// Before an insert into a full shared-memory array: both arrays to global
// memory for the rest of the batch (every thread calls it; kept out of line,
// off the batch loop's path).
template <int NT>
__device__ __noinline__ void fit_spill(FitSmem<NT>& S, const FitBlk* fa, const FitBlk* ua, FitBlk* gfa, FitBlk* gua,
                                       uint32_t gcap) {
    const uint32_t t = threadIdx.x;
    __syncthreads();
    for (uint32_t q = t; q < S.nf; q += NT) gfa[q] = fa[q];
    for (uint32_t q = t; q < S.nu; q += NT) gua[q] = ua[q];
    __syncthreads();
    if (t == 0) S.cap = gcap;
    __syncthreads();
}

// One arena's batch.  fa / ua: the arena's free and used arrays (capacity
// cap each); H: its header.
template <int NT>
__device__ void fit_arena(FitSmem<NT>& S, Arena& ar, FitHdr& H, FitBlk* gfa, FitBlk* gua, uint32_t gcap,
                          FitBlk* res, const uint64_t* frees, uint8_t* fstat, uint32_t f0, uint32_t f1,
                          const uint64_t* sizes, uint64_t* out, uint32_t a0, uint32_t a1) {
    const uint32_t t = threadIdx.x;
    const uint64_t A = ar.arena_bytes;
    const uint32_t lg = ar.lg, fit = H.fit;
    // the arrays in shared memory (res: 2 x FIT_RES entries) while they fit
    const uint32_t nf0 = H.nfree, nu0 = H.nused;
    bool resident = res != nullptr && nf0 < FIT_RES && nu0 < FIT_RES;
    FitBlk* fa = resident ? res : gfa;
    FitBlk* ua = resident ? res + FIT_RES : gua;
    const uint32_t cap = resident ? FIT_RES : gcap;
    auto spill = [&]() {
        fit_spill<NT>(S, fa, ua, gfa, gua, gcap);
        fa = gfa;
        ua = gua;
        resident = false;
    };
    if (resident) {
        for (uint32_t q = t; q < nf0; q += NT) fa[q] = gfa[q];
        for (uint32_t q = t; q < nu0; q += NT) ua[q] = gua[q];
    }
    if (t == 0) {
        S.nf = H.nfree;
        S.nu = H.nused;
        S.rover = H.rover;
        S.cap = cap;
        S.dirty = 1;
        S.err = 0;
        for (int q = 0; q < 6; ++q) S.cnt[q] = 0;
    }
    __syncthreads();
    // ---- frees (Algorithm 2), one by one
    for (uint32_t j = f0; j < f1; ++j) {
        __syncthreads();  // every thread is done with the previous free's broadcast values
        const uint64_t off = frees[j];
        const bool aligned = off < A && (off & ((1ull << lg) - 1)) == 0;
        const uint32_t g = aligned ? (uint32_t)(off >> lg) : 0u;
        uint32_t p = aligned ? fit_count_le<NT>(ua, S.nu, g, false) : 0u;
        if (t == 0) {
            uint32_t ok = 0, whole = 0, size = 0;
            if (aligned && p > 0) {
                const FitBlk it = ua[p - 1];
                if (g < it.a + it.z) {
                    ok = 1;
                    whole = it.a == g;
                    size = it.a + it.z - g;
                    if (!whole) ua[p - 1].z = g - it.a;  // partial deallocation: keep [start, g)
                }
            }
            S.v[0] = ok;
            S.v[1] = whole;
            S.v[2] = size;
            if (fstat) fstat[j] = ok ? 0 : 1;
            if (ok) {
                ++S.cnt[2];
                S.cnt[4] -= size;
            } else {
                ++S.cnt[3];
            }
        }
        __syncthreads();
        const uint32_t ok = S.v[0], whole = S.v[1], size = S.v[2];
        if (!ok) continue;
        if (whole) {
            fit_remove<NT>(ua, S.nu, p - 1);
            if (t == 0) --S.nu;
        }
        // coalesce with the free block ending at g and the one starting at g + size
        const uint32_t q = fit_count_le<NT>(fa, S.nf, g, false);
        if (t == 0) {
            const bool jl = q > 0 && fa[q - 1].a + fa[q - 1].z == g;
            const bool jr = q < S.nf && fa[q].a == g + size;
            uint32_t mode = 0;  // 0 insert, 1 left, 2 right, 3 both (4: insert after moving to global memory)
            if (jl && jr) {
                fa[q - 1].z += size + fa[q].z;
                mode = 3;
            } else if (jl) {
                fa[q - 1].z += size;
                mode = 1;
            } else if (jr) {
                fa[q].a = g;
                fa[q].z += size;
                mode = 2;
            }
            if (mode == 0 && resident && S.nf >= FIT_RES) mode = 4;  // the insert needs global memory first
            else if (mode == 0 && S.nf >= S.cap) S.err = ERR_LIST_WALK;  // cannot happen: cap > granules / 2
            S.v[3] = mode;
            S.dirty = 1;
        }
        __syncthreads();
        uint32_t mode = S.v[3];
        if (mode == 4) {
            spill();
            mode = 0;
        }
        if (mode == 3) {
            fit_remove<NT>(fa, S.nf, q);
            if (t == 0) --S.nf;
        } else if (mode == 0 && !S.err) {
            fit_insert<NT>(fa, S.nf, q, FitBlk{g, size});
            if (t == 0) ++S.nf;
        }
        __syncthreads();
    }
    // ---- allocations (Algorithm 1 on the fit's candidate), one by one; the
    // requests that the largest free block cannot serve fail together.
    // Sizes come NT at a time into shared memory; a window never crosses
    // such a group.
    for (uint32_t c0 = a0; c0 < a1; c0 += NT) {
    const uint32_t cend = a1 - c0 < (uint32_t)NT ? a1 : c0 + NT;
    __syncthreads();
    if (c0 + t < cend) S.wz[t] = sizes[c0 + t];
    __syncthreads();
    for (uint32_t i = c0; i < cend;) {
        if (S.dirty) fit_refresh_max<NT>(S, fa);
        const uint32_t n = cend - i;
        uint32_t sgr = 0;
        bool can = false;
        if (t < n) {
            const uint64_t sz = S.wz[i - c0 + t];
            if (sz != 0 && sz <= A) {
                sgr = (uint32_t)((sz + (1ull << lg) - 1) >> lg);
                can = sgr <= S.maxz;
            }
        }
        if (t == 0) S.v[4] = NT;
        __syncthreads();
        if (can) atomicMin(&S.v[4], t);
        __syncthreads();
        const uint32_t e = S.v[4] < n ? S.v[4] : n;  // first request that can be served
        if (t < e) out[i + t] = FAIL64;
        if (t == e) S.v[5] = sgr;
        if (t == 0) S.cnt[1] += e;
        __syncthreads();
        if (e < n) {
            const uint32_t s = S.v[5];
            const uint32_t c = fit_pick<NT>(S, fa, s, fit);
            if (c >= S.nf) {  // no candidate although the largest block fits: record, fail the request
                if (t == 0) {
                    S.err = ERR_EMPTY_HEAD;
                    out[i + e] = FAIL64;
                    ++S.cnt[1];
                    S.dirty = 1;
                }
                __syncthreads();
                i += e + 1;
                continue;
            }
            if (t == 0) {
                const FitBlk b = fa[c];
                S.v[6] = b.a;
                if (b.z > s) {
                    fa[c].a = b.a + s;  // the rest stays in place
                    fa[c].z = b.z - s;
                    S.v[3] = 0;
                } else {
                    S.v[3] = 1;
                }
                out[i + e] = (uint64_t)b.a << lg;
                S.rover = b.a + s;
                ++S.cnt[0];
                S.cnt[4] += s;
                S.cnt[5] += (int64_t)S.wz[i - c0 + e];
                S.dirty = 1;
            }
            __syncthreads();
            const uint32_t addr = S.v[6];
            if (S.v[3]) {
                fit_remove<NT>(fa, S.nf, c);
                if (t == 0) --S.nf;
            }
            if (resident && S.nu >= FIT_RES) spill();
            const uint32_t pu = fit_count_le<NT>(ua, S.nu, addr, false);
            if (S.nu < S.cap) {
                fit_insert<NT>(ua, S.nu, pu, FitBlk{addr, s});
                if (t == 0) ++S.nu;
            } else if (t == 0) {
                S.err = ERR_LIST_WALK;
            }
            __syncthreads();
        }
        i += e < n ? e + 1 : n;
    }
    }
    if (resident) {
        __syncthreads();
        for (uint32_t q = t; q < S.nf; q += NT) gfa[q] = fa[q];
        for (uint32_t q = t; q < S.nu; q += NT) gua[q] = ua[q];
    }
    if (t == 0) {
        H.nfree = S.nf;
        H.nused = S.nu;
        H.rover = S.rover;
        ar.alloc_ok += S.cnt[0];
        ar.alloc_fail += S.cnt[1];
        ar.free_ok += S.cnt[2];
        ar.free_fail += S.cnt[3];
        ar.used_g += S.cnt[4];
        ar.used_blocks = S.nu;
        ar.blocks = (int64_t)S.nu + S.nf;
        ar.requested += S.cnt[5];
        if (S.err && !ar.err) ar.err = S.err;
    }
    __syncthreads();
}
#endif

}  // namespace hba
