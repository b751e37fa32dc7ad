// hba_capi.cu -- C ABI of the header-free batched allocator (include/hba.h).
//
// Owns the device metadata of one or many arenas and launches the batch
// engine of hba_engine.cuh: one CTA per arena per batch.  No call here ever
// receives, reads or writes the managed arena itself.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "hba.h"
#include "hba_engine.cuh"
#include "hba_serve.cuh"
#include "hba_tlsf.cuh"
#include "hba_fits.cuh"
#include "hba_bitmask.cuh"

using hba::Arena;
using hba::Rec;

struct hba_s {
    int device = 0;
    uint32_t n_arenas = 0;
    uint64_t min_block = 0;
    uint32_t lg = 0;
    uint64_t total_granules = 0;
    Arena* d_arenas = nullptr;
    Rec* d_rec = nullptr;
    uint32_t* d_scr = nullptr;
    uint32_t* d_gi = nullptr;   // gathered records of a batch's frees (5 words each)
    uint64_t scr_frees = 0;     // scratch capacity in frees
    uint32_t max_batch = 0;     // single arena: frees per launch slice
    std::vector<Arena> h_init;  // initial headers (for reset)
    // staging for hba_step_host
    uint64_t* d_stage_f = nullptr;
    uint64_t* d_stage_s = nullptr;
    uint64_t* d_stage_o = nullptr;
    uint8_t* d_stage_st = nullptr;
    // pipelined host-buffer calls (hba_step_host_async,
    // hba_multi_step_host_async): two staging slots, used in turn, and three
    // internal streams -- input copies, the engine, result copies -- so that
    // one call's copies overlap its neighbours' kernels.  Made at create.
    struct Slot {
        uint64_t* f = nullptr;
        uint64_t* s = nullptr;
        uint64_t* o = nullptr;
        uint8_t* st = nullptr;
        uint32_t* fr = nullptr;  // many arenas: the two row-pointer arrays
        uint32_t* ar = nullptr;
        cudaEvent_t in = nullptr;    // inputs copied
        cudaEvent_t done = nullptr;  // batch applied
        cudaEvent_t out = nullptr;   // results copied back
        bool used = false;
    };
    Slot slot[2];
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    uint32_t next_slot = 0;
    uint64_t stage_allocs = 0;  // many arenas: allocations per host-buffer call (0: no staging)
    // launch shapes
    uint32_t threads = 0;       // single-arena CTA width (0: by batch size)
    uint32_t m_threads = 256;   // multi-arena CTA width
    uint32_t m_ctas = 0;        // multi-arena grid (0 = one CTA per arena)
    uint32_t smem_bytes = 0;    // dynamic shared memory per CTA (0 = automatic)
    uint32_t single_ctas = 0;   // single arena: CTAs of the batch cluster (0, 1 = prep grid + engine)
    uint64_t launches = 0;      // kernels this handle has launched
    // the last stream the handle's work went to, and an event after that work
    // (a call on another stream waits for it)
    cudaEvent_t ev = nullptr;
    cudaStream_t last = nullptr;
    bool have_last = false;
    uint64_t* d_largest = nullptr;
    uint32_t* d_extent = nullptr;  // per arena: end granule of the highest in-use block
    // two-level segregated fit (§5.2): per-arena lists and bitmaps, and their
    // initial state (for reset)
    int policy = HBA_POLICY_SEGFIT;
    hba::TlsfLists* d_tlsf = nullptr;
    std::vector<hba::TlsfLists> h_tlsf;
    // sequential fits (§3.1, §4): per-arena header, free and used arrays
    // (granules + 1 entries per arena each, at record base + arena index)
    hba::FitHdr* d_fhdr = nullptr;
    hba::FitBlk* d_fpool = nullptr;
    hba::FitBlk* d_upool = nullptr;
    std::vector<hba::FitHdr> h_fhdr;
    // bitmask pools (§3.2): per-pool header, free and start bitmaps
    hba::BmHdr* d_bmh = nullptr;
    uint64_t* d_bmF = nullptr;
    uint64_t* d_bmS = nullptr;
    std::vector<hba::BmHdr> h_bmh;
    uint32_t bm_wmax = 0;  // largest pool, in words
    // working buffers of hba_serve_run (queue, timing wheel, tick buffers),
    // kept between runs; a run that asks for a deeper queue or larger ticks
    // than any before replaces them
    static constexpr int SERVE_BUFS = 11;
    void* serve_buf[SERVE_BUFS] = {};
    uint32_t serve_qcap = 0, serve_batch = 0;
};

namespace {

#define HBA_CUDA_TRY(call)                         \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            (void)cudaGetLastError();              \
            return HBA_ERR_CUDA;                   \
        }                                          \
    } while (0)

// Dynamic shared memory holds the free-phase scratch of a batch (12 words
// per free) when it fits; otherwise the global scratch is used.  The single
// arena kernel takes everything the SM offers one CTA; the multi-arena
// kernel takes a per-CTA budget that leaves room for several CTAs per SM.
constexpr uint32_t MULTI_DYN_BYTES_DEFAULT = 24 * 1024;

// POL: the class layout (0 segregated fit; 1 two-level segregated fit,
// whose list heads and bitmaps are tl).
template <int NT, int POL = 0>
__global__ void __launch_bounds__(NT, 1) k_single(Arena* ar, Rec* rec, const uint64_t* frees, uint32_t nf,
                                               uint8_t* st, const uint64_t* sizes, uint32_t na,
                                               uint64_t* out, uint32_t* scr, const uint32_t* gi,
                                               uint32_t dyn_words, uint32_t prefilled, uint32_t self_gather,
                                               hba::TlsfLists* tl) {
    __shared__ hba::Smem<NT, POL> S;
    extern __shared__ __align__(16) uint32_t dyn[];
    // waits for the preceding prep grid (gathered records, pre-filled
    // failures) once it has read the arena header; or, with no prep grid,
    // gathers itself
    hba::StepArgs a{ar, rec, frees, nf, st, sizes, na, out, scr, gi, nf, prefilled,
                    self_gather ? hba::WAIT_NONE : hba::WAIT_GRID, 0, self_gather, tl};
    hba::arena_step<NT, POL>(S, a, dyn, dyn_words);
}

// Single arena as one thread-block cluster: CTA 0 runs the engine; CTAs
// 1..n-1 gather the records the frees need (hba::gather_words) straight into
// CTA 0's shared memory -- or into the global gather buffer when the free
// phase does not fit there -- and pre-fill out[] with HBA_FAIL, then arrive
// on the cluster barrier that CTA 0 waits on after reading the arena header.
// One launch per batch, and the gathered records need no second copy.
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_single_cl(Arena* ar, Rec* rec, const uint64_t* frees, uint32_t nf,
                                                  uint8_t* st, const uint64_t* sizes, uint32_t na,
                                                  uint64_t* out, uint32_t* scr, uint32_t* gi,
                                                  uint32_t dyn_words, uint32_t prefill, uint32_t staged) {
    __shared__ hba::Smem<NT> S;
    extern __shared__ __align__(16) uint32_t dyn[];
    uint32_t rank, nrank;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(nrank));
    if (rank == 0) {
        hba::cluster_arrive_relaxed();
        hba::StepArgs a{ar, rec, frees, nf, st, sizes, na, out, scr, gi, nf, prefill, hba::WAIT_CLUSTER, staged, 0};
        hba::arena_step<NT>(S, a, dyn, dyn_words);
        return;
    }
    const uint32_t t = (rank - 1) * NT + threadIdx.x, nth = (nrank - 1) * NT;
    const uint64_t A = ar->arena_bytes;
    const uint32_t G = ar->G, lg = ar->lg;
    // CTA 0's dynamic shared memory, in the cluster's shared window
    uint32_t eng;
    asm("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(eng) : "r"((uint32_t)__cvta_generic_to_shared(dyn)));
    for (uint32_t j = t; j < nf; j += nth) {
        uint32_t w[hba::GATHER_WORDS];
        hba::gather_words(rec, A, G, lg, frees[j], w);
#pragma unroll
        for (uint32_t q = 0; q < hba::GATHER_WORDS; ++q) {
            if (staged)
                asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(eng + 4u * (q * nf + j)), "r"(w[q]) : "memory");
            else
                gi[q * nf + j] = w[q];
        }
    }
    if (prefill && na) {
        uint32_t lo = 0;
        if ((uintptr_t)out & 15) {
            if (t == 0) out[0] = hba::FAIL64;
            lo = 1;
        }
        ulonglong2* o2 = reinterpret_cast<ulonglong2*>(out + lo);
        const uint32_t npair = (na - lo) / 2;
        for (uint32_t q = t; q < npair; q += nth) o2[q] = make_ulonglong2(hba::FAIL64, hba::FAIL64);
        if (((na - lo) & 1) && t == 0) out[na - 1] = hba::FAIL64;
    }
    hba::cluster_arrive_release();
    hba::cluster_wait();
}

template <int NT, int POL = 0>
__global__ void __launch_bounds__(NT) k_multi(Arena* ars, Rec* pool, const uint32_t* frow,
                                              const uint64_t* frees, uint8_t* st, const uint32_t* arow,
                                              const uint64_t* sizes, uint64_t* out, uint32_t* scr,
                                              const uint32_t* gi, uint32_t nf_total, uint32_t n_arenas,
                                              uint32_t dyn_words, uint32_t prefilled, hba::TlsfLists* tl) {
    __shared__ hba::Smem<NT, POL> S;
    extern __shared__ __align__(16) uint32_t dyn[];
    bool first = true;  // the first arena waits for the prep grid (after its header)
    for (uint32_t a = blockIdx.x; a < n_arenas; a += gridDim.x) {
        const uint32_t f0 = frow[a], f1 = frow[a + 1], a0 = arow[a], a1 = arow[a + 1];
        Arena* ar = ars + a;
        hba::StepArgs args{ar,
                           pool + ar->rec_base,
                           frees + f0,
                           f1 - f0,
                           st ? st + f0 : nullptr,
                           sizes + a0,
                           a1 - a0,
                           out + a0,
                           scr + (uint64_t)f0 * hba::SCRATCH_WORDS_PER_FREE,
                           gi + f0,
                           nf_total,
                           prefilled,
                           first ? hba::WAIT_GRID : hba::WAIT_NONE,
                           0,
                           0,
                           POL ? tl + a : nullptr};
        first = false;
        hba::arena_step<NT, POL>(S, args, dyn, dyn_words);
    }
}

// Warp mode: every warp of a CTA runs its own arenas (arena_step<32>, whose
// barriers are __syncwarp), W arenas per CTA at a time.  For many small
// arena batches, where a CTA per arena would spend its time in barriers.
// Segregated fit runs WPC warps per CTA; the two-level lists, whose per-arena
// shared state is four times larger (512 list heads and their cached
// records), run WPC_TL.
constexpr int WPC = 8;
#ifndef HBA_WPC_TL
#define HBA_WPC_TL 4
#endif
constexpr int WPC_TL = HBA_WPC_TL;
// MINB: at least this many CTAs per SM, a register budget for ptxas.  Two
// builds: 2 CTAs per SM (more registers, no spills) when the grid fits the
// SMs at that occupancy, 4 when it does not (more CTAs resident at once).
template <int MINB, int POL = 0, int W = WPC>
__global__ void __launch_bounds__(W * 32, MINB) k_multi_warp(Arena* ars, Rec* pool, const uint32_t* frow,
                                                        const uint64_t* frees, uint8_t* st, const uint32_t* arow,
                                                        const uint64_t* sizes, uint64_t* out, uint32_t* scr,
                                                        const uint32_t* gi, uint32_t nf_total, uint32_t n_arenas,
                                                        uint32_t warp_dyn_words, uint32_t prefilled,
                                                        hba::TlsfLists* tl) {
    __shared__ hba::Smem<32, POL> S[W];
    extern __shared__ __align__(16) uint32_t dyn[];
    bool first = true;  // the first arena waits for the prep grid (after its header)
    const uint32_t w = threadIdx.x >> 5;
    uint32_t* mine = dyn + (size_t)w * warp_dyn_words;
    for (uint32_t a = blockIdx.x * W + w; a < n_arenas; a += gridDim.x * W) {
        const uint32_t f0 = frow[a], f1 = frow[a + 1], a0 = arow[a], a1 = arow[a + 1];
        Arena* ar = ars + a;
        hba::StepArgs args{ar,
                           pool + ar->rec_base,
                           frees + f0,
                           f1 - f0,
                           st ? st + f0 : nullptr,
                           sizes + a0,
                           a1 - a0,
                           out + a0,
                           scr + (uint64_t)f0 * hba::SCRATCH_WORDS_PER_FREE,
                           gi + f0,
                           nf_total,
                           prefilled,
                           first ? hba::WAIT_GRID : hba::WAIT_NONE,
                           0,
                           0,
                           POL ? tl + a : nullptr};
        first = false;
        hba::arena_step<32, POL>(S[w], args, mine, warp_dyn_words);
    }
}

// Largest dynamic shared memory a CTA of k_single<NT> / k_multi<NT> can get.
struct SmemLimits {
    uint32_t single_dyn = 0, multi_dyn = 0;  // bytes
    uint32_t single_dyn_tl = 0;               // k_single<NT, 1> (two-level segregated fit)
    uint32_t multi_dyn_tl = 0;                // k_multi<NT, 1> (warp mode: k_multi_warp<., 1>, per warp)
    uint32_t alloc_words_tl = 0;
    uint32_t alloc_words = 0;                 // minimum dynamic words (alloc phase)
    uint32_t cluster_max = 0;                 // largest batch cluster that fits (0: none)
    uint32_t sms = 0;                         // SMs of the device (warp mode)
};

template <int NT>
SmemLimits set_smem_limits() {
    int dev = 0, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    SmemLimits L;
    L.alloc_words = hba::alloc_dyn_words<NT>();
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_single<NT>) == cudaSuccess) {
        L.single_dyn = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_single<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.single_dyn);
    }
    L.alloc_words_tl = hba::alloc_dyn_words<NT, 1>();
    if (cudaFuncGetAttributes(&fa, k_single<NT, 1>) == cudaSuccess) {
        L.single_dyn_tl = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_single<NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.single_dyn_tl);
    }
    if (cudaFuncGetAttributes(&fa, k_multi<NT>) == cudaSuccess) {
        L.multi_dyn = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_multi<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.multi_dyn);
    }
    if (cudaFuncGetAttributes(&fa, k_multi<NT, 1>) == cudaSuccess) {
        L.multi_dyn_tl = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_multi<NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.multi_dyn_tl);
    }
    if (NT >= 256 && cudaFuncGetAttributes(&fa, k_single_cl<NT>) == cudaSuccess) {
        const uint32_t dyn = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_single_cl<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        L.single_dyn = std::min(L.single_dyn, dyn);
        // the largest portable cluster of such CTAs that the device can hold
        for (uint32_t n = 8; n >= 2 && !L.cluster_max; n /= 2) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(n);
            cfg.blockDim = dim3(NT);
            cfg.dynamicSmemBytes = L.single_dyn;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = n;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, k_single_cl<NT>, &cfg) == cudaSuccess && nc > 0) L.cluster_max = n;
        }
        (void)cudaGetLastError();
    }
    return L;
}

SmemLimits g_limits[6];  // for 64, 128, 256, 512, 1024 threads; [5]: warp mode (32)
int limit_index(uint32_t threads) {
    switch (threads) {
        case 32: return 5;
        case 64: return 0;
        case 128: return 1;
        case 256: return 2;
        case 512: return 3;
        default: return 4;
    }
}

// warp mode: k_single<32> for one arena; k_multi_warp for many (per-warp budget)
SmemLimits set_smem_limits_warp() {
    int dev = 0, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    SmemLimits L;
    L.alloc_words = hba::alloc_dyn_words<32>();
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_single<32>) == cudaSuccess) {
        L.single_dyn = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_single<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.single_dyn);
    }
    L.alloc_words_tl = hba::alloc_dyn_words<32, 1>();
    if (cudaFuncGetAttributes(&fa, k_single<32, 1>) == cudaSuccess) {
        L.single_dyn_tl = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_single<32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.single_dyn_tl);
    }
    if (cudaFuncGetAttributes(&fa, k_multi_warp<2>) == cudaSuccess) {
        const uint32_t total = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_multi_warp<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
        cudaFuncSetAttribute(k_multi_warp<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
        L.multi_dyn = (total / WPC) & ~15u;  // per warp
    }
    if (cudaFuncGetAttributes(&fa, k_multi_warp<2, 1, WPC_TL>) == cudaSuccess) {
        const uint32_t total = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
        cudaFuncSetAttribute(k_multi_warp<2, 1, WPC_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
        cudaFuncSetAttribute(k_multi_warp<4, 1, WPC_TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total);
        L.multi_dyn_tl = (total / WPC_TL) & ~15u;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    L.sms = (uint32_t)sms;
    return L;
}

// The prep grid of a batch, on many SMs: gathers the records every free
// needs (hba::gather_free, one thread per free; one SM alone could keep too
// few random loads in flight) and pre-fills out[0..na) with HBA_FAIL, so that
// the allocator kernel that follows (programmatic dependent launch) stores
// only successes.  frow (multi-arena) maps a free to its arena.
__global__ void k_prep(const Arena* ars, const Rec* pool, const uint32_t* frow, uint32_t n_arenas,
                       const uint64_t* frees, uint32_t nf, uint32_t* gi, uint64_t* out, uint32_t na) {
    asm volatile("griddepcontrol.launch_dependents;");
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (uint32_t j = t0; j < nf; j += nth) {
        uint32_t a = 0;
        if (frow) {  // last arena whose first free is <= j
            uint32_t lo = 0, hi = n_arenas;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) / 2;
                if (frow[mid] <= j) lo = mid;
                else hi = mid;
            }
            a = lo;
        }
        const Arena& ar = ars[a];
        hba::gather_free(pool + ar.rec_base, ar.arena_bytes, ar.G, ar.lg, frees[j], gi, nf, j);
    }
    if (out && na) {
        uint32_t lo = 0;
        if ((uintptr_t)out & 15) {
            if (t0 == 0) out[0] = hba::FAIL64;
            lo = 1;
        }
        ulonglong2* o2 = reinterpret_cast<ulonglong2*>(out + lo);
        const uint32_t npair = (na - lo) / 2;
        for (uint32_t q = t0; q < npair; q += nth) o2[q] = make_ulonglong2(hba::FAIL64, hba::FAIL64);
        if (((na - lo) & 1) && t0 == 0) out[na - 1] = hba::FAIL64;
    }
}

// Allocation batches at least this large get their failures pre-filled.
constexpr uint32_t PREFILL_MIN = 2048;
// Single-arena batches of at most this many frees and this many allocations
// run on 128-thread CTAs when the handle leaves the width automatic; larger
// ones on 1,024.
constexpr uint32_t AUTO_SMALL_BATCH = 256;
// Batches with at most this many frees (and no pre-filling) are gathered by
// the engine CTA itself: one launch instead of two.
#ifndef HBA_SELF_GATHER_MAX
#define HBA_SELF_GATHER_MAX 512
#endif
constexpr uint32_t SELF_GATHER_MAX = HBA_SELF_GATHER_MAX;

// Launch the prep grid if the batch needs one; returns whether out[] is
// pre-filled.  *pdl is set when the next launch may depend on it.
// Extent of every arena: the end (in granules) of its highest in-use block,
// 0 when none is in use.  The start granule of every in-use block holds an
// ST_USED record and no other granule does, so this is a max-reduction over
// the record table.  A CTA takes a tile of 64 x blockDim granules, a thread
// every blockDim-th granule of it (coalesced); a thread finds the arena of
// its first granule by binary search over the record bases (contiguous,
// ascending) and steps to the next arena at a boundary.  ext[] must be zero.
__global__ void k_extent(const Arena* ars, const Rec* pool, uint32_t n_arenas, uint64_t total, uint32_t* ext) {
    const uint64_t T = 64ull * blockDim.x;
    for (uint64_t t0 = (uint64_t)blockIdx.x * T; t0 < total; t0 += (uint64_t)gridDim.x * T) {
        uint64_t q = t0 + threadIdx.x;
        if (q >= total) continue;
        uint32_t lo = 0, hi = n_arenas - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) / 2;
            if (ars[mid].rec_base <= q) lo = mid;
            else hi = mid - 1;
        }
        uint32_t a = lo;
        uint64_t base = ars[a].rec_base, end = base + ars[a].G;
        uint32_t best = 0;
        const uint64_t stop = t0 + T < total ? t0 + T : total;
        for (; q < stop; q += blockDim.x) {
            while (q >= end && a + 1 < n_arenas) {
                if (best) atomicMax(&ext[a], best);
                best = 0;
                ++a;
                base = ars[a].rec_base;
                end = base + ars[a].G;
            }
            const uint32_t x = pool[q].x;
            if (hba::st_of(x) == hba::ST_USED) {
                const uint32_t e = (uint32_t)(q - base) + hba::sz_of(x);
                if (e > best) best = e;
            }
        }
        if (best) atomicMax(&ext[a], best);
    }
}

// Sequential fits: one CTA per arena, the grid striding over the arenas.
// frow / arow: each arena's row offsets into frees / sizes (n_arenas + 1
// entries), or null for a single arena, whose requests are frees[0, nf) and
// sizes[0, na).
template <int NT>
__global__ void __launch_bounds__(NT) k_fits(Arena* ars, hba::FitHdr* hdr, hba::FitBlk* fpool, hba::FitBlk* upool,
                                            uint32_t n_arenas, const uint32_t* frow, const uint64_t* frees,
                                            uint8_t* fstat, uint32_t nf, const uint32_t* arow, const uint64_t* sizes,
                                            uint64_t* out, uint32_t na, uint32_t res_words) {
    __shared__ hba::FitSmem<NT> S;
    extern __shared__ __align__(16) hba::FitBlk fit_res[];  // 2 x FIT_RES entries, or none
    for (uint32_t a = blockIdx.x; a < n_arenas; a += gridDim.x) {
        Arena& ar = ars[a];
        const uint64_t base = ar.rec_base + a;
        const uint32_t f0 = frow ? frow[a] : 0u, f1 = frow ? frow[a + 1] : nf;
        const uint32_t a0 = arow ? arow[a] : 0u, a1 = arow ? arow[a + 1] : na;
        hba::fit_arena<NT>(S, ar, hdr[a], fpool + base, upool + base, ar.G + 1, res_words ? fit_res : nullptr, frees,
                           fstat, f0, f1, sizes, out, a0, a1);
    }
}

// Bitmask pools: one CTA per pool, both bitmaps in dynamic shared memory
// (2 x bm_wmax words).  frow / arow as for k_fits.
template <int NT>
__global__ void __launch_bounds__(NT) k_bitmask(Arena* ars, hba::BmHdr* hdr, uint64_t* gF, uint64_t* gS,
                                               uint32_t n_arenas, uint32_t wmax, const uint32_t* frow,
                                               const uint64_t* frees, uint8_t* fstat, uint32_t nf,
                                               const uint32_t* arow, const uint64_t* sizes, uint64_t* out,
                                               uint32_t na) {
    __shared__ hba::BmSmem<NT> S_;
    extern __shared__ __align__(16) uint64_t bm_dyn[];
    for (uint32_t a = blockIdx.x; a < n_arenas; a += gridDim.x) {
        const uint32_t f0 = frow ? frow[a] : 0u, f1 = frow ? frow[a + 1] : nf;
        const uint32_t a0 = arow ? arow[a] : 0u, a1 = arow ? arow[a + 1] : na;
        hba::BmHdr& H = hdr[a];
        hba::bm_pool<NT>(S_, ars[a], H, gF + H.wbase, gS + H.wbase, bm_dyn, bm_dyn + wmax, frees, fstat, f0, f1,
                         sizes, out, a0, a1);
    }
}

// Initial bitmaps: every unit free (bits past the pool's end clear), no starts.
__global__ void k_bm_init(const Arena* ars, const hba::BmHdr* hdr, uint64_t* gF, uint64_t* gS, uint32_t n_arenas) {
    for (uint32_t a = blockIdx.x; a < n_arenas; a += gridDim.x) {
        const uint32_t N = ars[a].G, W = hdr[a].words;
        uint64_t* F = gF + hdr[a].wbase;
        uint64_t* S = gS + hdr[a].wbase;
        for (uint32_t w = threadIdx.x; w < W; w += blockDim.x) {
            const uint32_t lo = w << 6;
            F[w] = N - lo >= 64 ? ~0ull : (1ull << (N - lo)) - 1ull;
            S[w] = 0;
        }
    }
}

// Space report of the bitmask pools: longest free run (bytes), extent (units:
// one past the highest in-use unit), and the block count (in-use blocks +
// free runs) into the arena header.
__global__ void k_bm_space(Arena* ars, const hba::BmHdr* hdr, const uint64_t* gF, const uint64_t* gS,
                           uint32_t n_arenas, uint64_t* largest, uint32_t* extent) {
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_arenas) return;
    const uint32_t N = ars[a].G;
    const uint64_t* F = gF + hdr[a].wbase;
    const uint64_t* S = gS + hdr[a].wbase;
    uint32_t run = 0, longest = 0, runs = 0, used = 0, top = 0;
    for (uint32_t u = 0; u < N; ++u) {
        const uint64_t fw = F[u >> 6];
        used += (uint32_t)((S[u >> 6] >> (u & 63)) & 1ull);
        if ((fw >> (u & 63)) & 1ull) {
            if (run == 0) ++runs;
            ++run;
            if (run > longest) longest = run;
        } else {
            run = 0;
            top = u + 1;
        }
    }
    largest[a] = (uint64_t)longest << ars[a].lg;
    extent[a] = top;
    ars[a].blocks = (int64_t)used + runs;
}

// Initial free arrays of the sequential fits: one block [0, G) per arena.
__global__ void k_fits_init(const Arena* ars, hba::FitBlk* fpool, uint32_t n_arenas) {
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_arenas) return;
    fpool[ars[a].rec_base + a] = hba::FitBlk{0u, ars[a].G};
}

// Space report of the sequential fits: largest free block (bytes) and
// extent (granules: the end of the last used block, the used array being
// sorted by address).
__global__ void k_fits_space(const Arena* ars, const hba::FitHdr* hdr, const hba::FitBlk* fpool,
                             const hba::FitBlk* upool, uint32_t n_arenas, uint64_t* largest, uint32_t* extent) {
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_arenas) return;
    const uint64_t base = ars[a].rec_base + a;
    uint32_t m = 0;
    for (uint32_t i = 0; i < hdr[a].nfree; ++i) m = max(m, fpool[base + i].z);
    largest[a] = (uint64_t)m << ars[a].lg;
    const uint32_t nu = hdr[a].nused;
    extent[a] = nu ? upool[base + nu - 1].a + upool[base + nu - 1].z : 0u;
}

// Largest free block of every TLSF arena: the highest non-empty list is
// walked (bounded by the arena's block count).
__global__ void k_largest_tlsf(const Arena* ars, const hba::TlsfLists* lists, const Rec* pool, uint32_t n_arenas,
                               uint64_t* out) {
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_arenas) return;
    const Arena& ar = ars[a];
    const hba::TlsfLists& L = lists[a];
    uint64_t best = 0;
    if (L.flmask) {
        const uint32_t f = hba::flog2(L.flmask);
        const uint32_t k = f * hba::TL_SL + hba::flog2(L.slmask[f]);
        const Rec* rec = pool + ar.rec_base;
        uint64_t guard = 0;
        for (uint32_t h = L.heads[k]; h != hba::NIL && guard <= (uint64_t)ar.blocks; ++guard) {
            const uint32_t sz = hba::sz_of(rec[h].x);
            if (sz > best) best = sz;
            h = rec[h].z;
        }
    }
    out[a] = best << ar.lg;
}

bool launch_prep(hba_t h, const uint32_t* frow, const uint64_t* frees, uint32_t nf, uint32_t* gi, uint64_t* out,
                 uint32_t na, cudaStream_t s, bool* pdl);

// Launch with a programmatic dependency on the preceding kernel of the stream.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), uint32_t grid, uint32_t block, uint32_t dyn, cudaStream_t s,
                       bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Write the initial record of every arena (one free block spanning it).
__global__ void k_init_records(const Arena* ars, Rec* pool, uint32_t n_arenas) {
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_arenas) {
        const Arena& ar = ars[a];
        const Rec r{hba::mkx(ar.G, hba::ST_FREE), hba::NIL, hba::NIL, hba::NIL};
        *reinterpret_cast<uint4*>(pool + ar.rec_base) = make_uint4(r.x, r.y, r.z, r.w);
    }
}

// Largest free block of every arena: its highest non-empty class's list is
// walked (bounded by the arena's block count).
__global__ void k_largest(const Arena* ars, const Rec* pool, uint32_t n_arenas, uint64_t* out) {
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_arenas) return;
    const Arena& ar = ars[a];
    uint64_t best = 0;
    if (ar.mask) {
        const uint32_t b = 63u - (uint32_t)__clzll((long long)ar.mask);
        const Rec* rec = pool + ar.rec_base;
        uint64_t guard = 0;
        for (uint32_t h = ar.heads[b]; h != hba::NIL && guard <= (uint64_t)ar.blocks; ++guard) {
            const uint32_t sz = hba::sz_of(rec[h].x);
            if (sz > best) best = sz;
            h = rec[h].z;
        }
    }
    out[a] = best << ar.lg;
}

bool launch_prep(hba_t h, const uint32_t* frow, const uint64_t* frees, uint32_t nf, uint32_t* gi, uint64_t* out,
                 uint32_t na, cudaStream_t s, bool* pdl) {
    const bool fill = na >= PREFILL_MIN;
    *pdl = false;
    if (!nf && !fill) return false;
    const uint32_t work = std::max(nf, fill ? na / 2 : 0u);
    const uint32_t blocks = std::max(1u, std::min<uint32_t>((work + 127) / 128, 2048));
    k_prep<<<blocks, 128, 0, s>>>(h->d_arenas, h->d_rec, frow, h->n_arenas, frees, nf, gi,
                                  fill ? out : nullptr, fill ? na : 0);
    ++h->launches;
    *pdl = true;
    return fill;
}

// Launch a batch cluster of n CTAs (one cluster).
template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(void (*k)(KArgs...), uint32_t n, uint32_t block, uint32_t dyn, cudaStream_t s,
                           Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = n;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// One batch of a single arena: the prep grid and the engine kernel, or, when
// the handle asks for a cluster of 2..8 CTAs and the device holds one, a
// batch cluster (engine + gathering CTAs).  gi / scr: the gather buffer and
// the free-phase scratch to use.
// One batch of a single-arena handle: the prep grid when the batch needs it,
// then the engine (POL: the class layout of the handle's policy).
template <int POL>
hba_status_t launch_single_p(hba_t h, const uint64_t* frees, uint32_t nf, uint8_t* st, const uint64_t* sizes,
                             uint32_t na, uint64_t* out, cudaStream_t s, uint32_t* gi, uint32_t* scr) {
    hba::TlsfLists* tl = POL ? h->d_tlsf : nullptr;
    Arena* ar = h->d_arenas;
    Rec* rec = h->d_rec;
    // CTA width: the handle's, or by batch size (small batches pay less per
    // barrier with fewer threads)
    const uint32_t nt = h->threads ? h->threads : (std::max(nf, na) <= AUTO_SMALL_BATCH ? 128u : 1024u);
    const int li = limit_index(nt);
    const SmemLimits& L = g_limits[li];
    const uint32_t maxdyn = POL ? L.single_dyn_tl : L.single_dyn;
    const uint32_t base = 4 * (POL ? L.alloc_words_tl : L.alloc_words);
    uint32_t dyn;
    if (h->smem_bytes) {
        dyn = std::max(base, std::min(h->smem_bytes, maxdyn));
    } else {
        // what this batch's free phase keeps in shared memory (if it fits),
        // so that L1 keeps the rest
        const uint64_t hot = 4ull * hba::free_smem_words(nf);
        dyn = hot <= maxdyn ? (uint32_t)std::max<uint64_t>(hot, base) : base;
    }
    dyn = (dyn + 15u) & ~15u;
    const uint32_t dw = dyn / 4;
    const bool fill = na >= PREFILL_MIN;
    cudaError_t e;
    if (POL == 0 && nt >= 256 && h->single_ctas >= 2 && L.cluster_max >= 2 && (nf || fill)) {
        const uint32_t ncl = std::min(h->single_ctas, L.cluster_max);
        const uint32_t staged = nf && hba::stage_fits(nf, dw) ? 1u : 0u;
        const uint32_t pf = fill ? 1u : 0u;
        switch (nt) {
            case 256: e = launch_cluster(k_single_cl<256>, ncl, 256, dyn, s, ar, rec, frees, nf, st, sizes, na, out, scr, gi, dw, pf, staged); break;
            case 512: e = launch_cluster(k_single_cl<512>, ncl, 512, dyn, s, ar, rec, frees, nf, st, sizes, na, out, scr, gi, dw, pf, staged); break;
            default: e = launch_cluster(k_single_cl<1024>, ncl, 1024, dyn, s, ar, rec, frees, nf, st, sizes, na, out, scr, gi, dw, pf, staged); break;
        }
        if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return HBA_ERR_CUDA;
        ++h->launches;
        return HBA_OK;
    }
    // small batches without pre-filling: the engine gathers its frees itself
    // (one launch); otherwise the prep grid gathers on many SMs
    const uint32_t self = nf <= SELF_GATHER_MAX && !fill ? 1u : 0u;
    bool pdl = false;
    const bool pre = self ? false : launch_prep(h, nullptr, frees, nf, gi, out, na, s, &pdl);
    if (cudaGetLastError() != cudaSuccess) return HBA_ERR_CUDA;
    const uint32_t pf = pre ? 1u : 0u;
    const uint32_t* g = gi;
    switch (nt) {
        case 32: e = launch_pdl(k_single<32, POL>, 1, 32, dyn, s, pdl, ar, rec, frees, nf, st, sizes, na, out, scr, g, dw, pf, self, tl); break;
        case 64: e = launch_pdl(k_single<64, POL>, 1, 64, dyn, s, pdl, ar, rec, frees, nf, st, sizes, na, out, scr, g, dw, pf, self, tl); break;
        case 128: e = launch_pdl(k_single<128, POL>, 1, 128, dyn, s, pdl, ar, rec, frees, nf, st, sizes, na, out, scr, g, dw, pf, self, tl); break;
        case 256: e = launch_pdl(k_single<256, POL>, 1, 256, dyn, s, pdl, ar, rec, frees, nf, st, sizes, na, out, scr, g, dw, pf, self, tl); break;
        case 512: e = launch_pdl(k_single<512, POL>, 1, 512, dyn, s, pdl, ar, rec, frees, nf, st, sizes, na, out, scr, g, dw, pf, self, tl); break;
        default: e = launch_pdl(k_single<1024, POL>, 1, 1024, dyn, s, pdl, ar, rec, frees, nf, st, sizes, na, out, scr, g, dw, pf, self, tl); break;
    }
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return HBA_ERR_CUDA;
    ++h->launches;
    return HBA_OK;
}

hba_status_t launch_single(hba_t h, const uint64_t* frees, uint32_t nf, uint8_t* st, const uint64_t* sizes,
                           uint32_t na, uint64_t* out, cudaStream_t s, uint32_t* gi, uint32_t* scr) {
    return h->policy == HBA_POLICY_TLSF ? launch_single_p<1>(h, frees, nf, st, sizes, na, out, s, gi, scr)
                                        : launch_single_p<0>(h, frees, nf, st, sizes, na, out, s, gi, scr);
}

bool is_fit(int policy) {
    return policy == HBA_POLICY_FIRST_FIT || policy == HBA_POLICY_NEXT_FIT || policy == HBA_POLICY_BEST_FIT;
}

// A sequential-fit batch: one CTA of FIT_NT threads per arena.
#ifndef HBA_FIT_NT
#define HBA_FIT_NT 256
#endif
constexpr int FIT_NT = HBA_FIT_NT;
hba_status_t launch_fits(hba_t h, const uint32_t* frow, const uint64_t* frees, uint32_t nf, uint8_t* st,
                         const uint32_t* arow, const uint64_t* sizes, uint32_t na, uint64_t* out, cudaStream_t s) {
    const uint32_t n = h->n_arenas;
    const uint32_t sms = g_limits[5].sms ? g_limits[5].sms : 152u;
    const uint32_t grid = std::min(n, 8u * sms);
    const uint32_t res = (uint32_t)(2 * sizeof(hba::FitBlk) * hba::FIT_RES);  // shared-memory arrays
    k_fits<FIT_NT><<<grid, FIT_NT, res, s>>>(h->d_arenas, h->d_fhdr, h->d_fpool, h->d_upool, n, frow, frees, st, nf,
                                             arow, sizes, out, na, res / 4);
    ++h->launches;
    return cudaGetLastError() == cudaSuccess ? HBA_OK : HBA_ERR_CUDA;
}

// A bitmask batch: one CTA of BM_NT threads per pool.
#ifndef HBA_BM_NT
#define HBA_BM_NT 256
#endif
constexpr int BM_NT = HBA_BM_NT;
hba_status_t launch_bitmask(hba_t h, const uint32_t* frow, const uint64_t* frees, uint32_t nf, uint8_t* st,
                            const uint32_t* arow, const uint64_t* sizes, uint32_t na, uint64_t* out,
                            cudaStream_t s) {
    const uint32_t n = h->n_arenas;
    const uint32_t sms = g_limits[5].sms ? g_limits[5].sms : 152u;
    const uint32_t grid = std::min(n, 4u * sms);
    const uint32_t dyn = 16u * h->bm_wmax;
    k_bitmask<BM_NT><<<grid, BM_NT, dyn, s>>>(h->d_arenas, h->d_bmh, h->d_bmF, h->d_bmS, n, h->bm_wmax, frow, frees,
                                              st, nf, arow, sizes, out, na);
    ++h->launches;
    return cudaGetLastError() == cudaSuccess ? HBA_OK : HBA_ERR_CUDA;
}

hba_status_t step_impl(hba_t h, const uint64_t* frees, uint32_t nf, uint8_t* st, const uint64_t* sizes,
                       uint32_t na, uint64_t* out, cudaStream_t s) {
    if (!h || h->n_arenas != 1) return HBA_ERR_INVALID_ARGUMENT;
    if ((nf && !frees) || (na && (!sizes || !out))) return HBA_ERR_INVALID_ARGUMENT;
    if (is_fit(h->policy)) {
        if (nf == 0 && na == 0) return HBA_OK;
        return launch_fits(h, nullptr, frees, nf, st, nullptr, sizes, na, out, s);
    }
    if (h->policy == HBA_POLICY_BITMASK) {
        if (nf == 0 && na == 0) return HBA_OK;
        return launch_bitmask(h, nullptr, frees, nf, st, nullptr, sizes, na, out, s);
    }
    // frees beyond the scratch capacity go in consecutive slices (exact:
    // frees apply one by one in index order).  Slicing at what one free
    // phase keeps in shared memory was measured slower on the fragmentation
    // workload (16,384 frees: four sliced launch pairs against one free
    // phase on global scratch), so it is not done.
    while (nf > h->max_batch) {
        hba_status_t r = launch_single(h, frees, h->max_batch, st, nullptr, 0, nullptr, s, h->d_gi, h->d_scr);
        if (r != HBA_OK) return r;
        frees += h->max_batch;
        if (st) st += h->max_batch;
        nf -= h->max_batch;
    }
    if (nf == 0 && na == 0) return HBA_OK;
    return launch_single(h, frees, nf, st, sizes, na, out, s, h->d_gi, h->d_scr);
}

// The staging slots and streams of the pipelined host-buffer calls: nf_cap
// frees and na_cap allocations a slot, and (many arenas) rows row pointers
// of each kind.
hba_status_t make_pipeline(hba_t h, uint64_t nf_cap, uint64_t na_cap, uint64_t rows) {
    nf_cap = std::max<uint64_t>(nf_cap, 1);
    na_cap = std::max<uint64_t>(na_cap, 1);
    for (hba_s::Slot& q : h->slot) {
        if (cudaMalloc(&q.f, 8 * nf_cap) != cudaSuccess || cudaMalloc(&q.s, 8 * na_cap) != cudaSuccess ||
            cudaMalloc(&q.o, 8 * na_cap) != cudaSuccess || cudaMalloc(&q.st, nf_cap) != cudaSuccess)
            return HBA_ERR_OUT_OF_MEMORY;
        if (rows && (cudaMalloc(&q.fr, 4 * rows) != cudaSuccess || cudaMalloc(&q.ar, 4 * rows) != cudaSuccess))
            return HBA_ERR_OUT_OF_MEMORY;
        HBA_CUDA_TRY(cudaEventCreateWithFlags(&q.in, cudaEventDisableTiming));
        HBA_CUDA_TRY(cudaEventCreateWithFlags(&q.done, cudaEventDisableTiming));
        HBA_CUDA_TRY(cudaEventCreateWithFlags(&q.out, cudaEventDisableTiming));
    }
    HBA_CUDA_TRY(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
    HBA_CUDA_TRY(cudaStreamCreateWithFlags(&h->s_run, cudaStreamNonBlocking));
    HBA_CUDA_TRY(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
    return HBA_OK;
}

hba_status_t alloc_meta(hba_t h, const std::vector<Arena>& init, uint64_t scr_frees, uint32_t stage) {
    g_limits[0] = set_smem_limits<64>();
    g_limits[1] = set_smem_limits<128>();
    g_limits[2] = set_smem_limits<256>();
    g_limits[3] = set_smem_limits<512>();
    g_limits[4] = set_smem_limits<1024>();
    g_limits[5] = set_smem_limits_warp();
    HBA_CUDA_TRY(cudaGetLastError());
    h->h_init = init;
    h->n_arenas = (uint32_t)init.size();
    HBA_CUDA_TRY(cudaGetDevice(&h->device));
    if (cudaMalloc(&h->d_arenas, sizeof(Arena) * init.size()) != cudaSuccess) return HBA_ERR_OUT_OF_MEMORY;
    if (cudaMalloc(&h->d_rec, sizeof(Rec) * h->total_granules) != cudaSuccess) return HBA_ERR_OUT_OF_MEMORY;
    h->scr_frees = scr_frees;
    if (cudaMalloc(&h->d_scr, 4ull * hba::SCRATCH_WORDS_PER_FREE * std::max<uint64_t>(scr_frees, 1)) != cudaSuccess)
        return HBA_ERR_OUT_OF_MEMORY;
    if (cudaMalloc(&h->d_gi, 4ull * hba::GATHER_WORDS * std::max<uint64_t>(scr_frees, 1)) != cudaSuccess)
        return HBA_ERR_OUT_OF_MEMORY;
    if (cudaMalloc(&h->d_largest, sizeof(uint64_t) * init.size()) != cudaSuccess) return HBA_ERR_OUT_OF_MEMORY;
    if (cudaMalloc(&h->d_extent, sizeof(uint32_t) * init.size()) != cudaSuccess) return HBA_ERR_OUT_OF_MEMORY;
    HBA_CUDA_TRY(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming));
    if (stage) {
        if (cudaMalloc(&h->d_stage_f, 8ull * stage) != cudaSuccess ||
            cudaMalloc(&h->d_stage_s, 8ull * stage) != cudaSuccess ||
            cudaMalloc(&h->d_stage_o, 8ull * stage) != cudaSuccess ||
            cudaMalloc(&h->d_stage_st, stage) != cudaSuccess)
            return HBA_ERR_OUT_OF_MEMORY;
        return make_pipeline(h, stage, stage, 0);
    }
    return HBA_OK;
}

// Orders a call's work after the handle's previous work when the streams
// differ (an event recorded after every call); does nothing while the stream
// is being captured.
struct StreamOrder {
    hba_t h;
    cudaStream_t s;
    bool on = false;
    StreamOrder(hba_t h_, cudaStream_t s_) : h(h_), s(s_) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (!h || !h->ev || cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        on = true;
        if (h->have_last && h->last != s) cudaStreamWaitEvent(s, h->ev, 0);
    }
    ~StreamOrder() {
        if (!on) return;
        cudaEventRecord(h->ev, s);
        h->last = s;
        h->have_last = true;
    }
};

hba_status_t reset_impl(hba_t h, cudaStream_t s) {
    HBA_CUDA_TRY(cudaMemsetAsync(h->d_rec, 0, sizeof(Rec) * h->total_granules, s));
    if (h->d_tlsf)
        HBA_CUDA_TRY(cudaMemcpyAsync(h->d_tlsf, h->h_tlsf.data(), sizeof(hba::TlsfLists) * h->n_arenas,
                                     cudaMemcpyHostToDevice, s));
    HBA_CUDA_TRY(cudaMemcpyAsync(h->d_arenas, h->h_init.data(), sizeof(Arena) * h->n_arenas,
                                 cudaMemcpyHostToDevice, s));
    k_init_records<<<(h->n_arenas + 255) / 256, 256, 0, s>>>(h->d_arenas, h->d_rec, h->n_arenas);
    ++h->launches;
    if (h->d_bmh) {  // after the arena headers, whose sizes it reads
        HBA_CUDA_TRY(cudaMemcpyAsync(h->d_bmh, h->h_bmh.data(), sizeof(hba::BmHdr) * h->n_arenas,
                                     cudaMemcpyHostToDevice, s));
        k_bm_init<<<std::min<uint32_t>(h->n_arenas, 1024u), 256, 0, s>>>(h->d_arenas, h->d_bmh, h->d_bmF, h->d_bmS,
                                                                        h->n_arenas);
        ++h->launches;
    }
    if (h->d_fhdr) {  // after the arena headers, whose record bases it reads
        HBA_CUDA_TRY(cudaMemcpyAsync(h->d_fhdr, h->h_fhdr.data(), sizeof(hba::FitHdr) * h->n_arenas,
                                     cudaMemcpyHostToDevice, s));
        k_fits_init<<<(h->n_arenas + 255) / 256, 256, 0, s>>>(h->d_arenas, h->d_fpool, h->n_arenas);
        ++h->launches;
    }
    HBA_CUDA_TRY(cudaGetLastError());
    return HBA_OK;
}

void free_all(hba_t h) {
    cudaFree(h->d_arenas);
    cudaFree(h->d_rec);
    cudaFree(h->d_scr);
    cudaFree(h->d_gi);
    cudaFree(h->d_largest);
    cudaFree(h->d_extent);
    cudaFree(h->d_tlsf);
    cudaFree(h->d_fhdr);
    cudaFree(h->d_fpool);
    cudaFree(h->d_upool);
    cudaFree(h->d_bmh);
    cudaFree(h->d_bmF);
    cudaFree(h->d_bmS);
    cudaFree(h->d_stage_f);
    cudaFree(h->d_stage_s);
    cudaFree(h->d_stage_o);
    cudaFree(h->d_stage_st);
    for (hba_s::Slot& q : h->slot) {
        cudaFree(q.f);
        cudaFree(q.s);
        cudaFree(q.o);
        cudaFree(q.st);
        cudaFree(q.fr);
        cudaFree(q.ar);
        if (q.in) cudaEventDestroy(q.in);
        if (q.done) cudaEventDestroy(q.done);
        if (q.out) cudaEventDestroy(q.out);
    }
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_run) cudaStreamDestroy(h->s_run);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->ev) cudaEventDestroy(h->ev);
    for (void*& p : h->serve_buf) {
        cudaFree(p);
        p = nullptr;
    }
}

bool check_geometry(uint64_t arena_bytes, uint64_t min_block, uint32_t* lg, uint64_t* a) {
    if (min_block < 8 || (min_block & (min_block - 1))) return false;
    *lg = (uint32_t)__builtin_ctzll(min_block);
    *a = arena_bytes - arena_bytes % min_block;
    const uint64_t G = *a >> *lg;
    return G >= 1 && G <= hba::MAX_GRANULES;
}

// ---- the serving loop ----------------------------------------------------
#ifndef HBA_SERVE_NT
#define HBA_SERVE_NT 256
#endif
constexpr int SERVE_NT = HBA_SERVE_NT;
__global__ void __launch_bounds__(SERVE_NT, 1) k_serve(hba::ServeArgs g, uint32_t dyn_words) {
    __shared__ hba::Smem<SERVE_NT> S;
    __shared__ hba::ServeSmem<SERVE_NT> Q;
    extern __shared__ __align__(16) uint32_t dyn[];
    hba::serve_loop<SERVE_NT>(S, Q, g, dyn, dyn_words);
}

static_assert(sizeof(hba_arrival_t) == sizeof(hba::Arrival), "arrival layout");
static_assert(sizeof(hba_served_t) == sizeof(hba::Served), "served layout");
static_assert(sizeof(hba_serve_report_t) == sizeof(hba::ServeCtl), "report layout");
static_assert(offsetof(hba_serve_report_t, idle_ticks) == offsetof(hba::ServeCtl, idle_ticks) &&
                  offsetof(hba_serve_report_t, status) == offsetof(hba::ServeCtl, status) &&
                  offsetof(hba_serve_report_t, log_words) == offsetof(hba::ServeCtl, log_words),
              "report field order");
static_assert(offsetof(hba_arrival_t, hold_ns) == offsetof(hba::Arrival, hold_ns) &&
                  offsetof(hba_served_t, t_free_ns) == offsetof(hba::Served, t_free_ns),
              "arrival / served field order");
static_assert(HBA_REJECTED == hba::REJECTED64, "rejected marker");

hba_status_t serve_impl(hba_t h, const hba_arrival_t* arr, uint64_t n, hba_served_t* served, uint32_t* log,
                        uint64_t log_cap, const hba_serve_config_t* cfg, hba_serve_report_t* rep, cudaStream_t s) {
    if (!h || h->n_arenas != 1 || !rep || (n && (!arr || !served)) || n >= 0xFFFFFFFFull || (log_cap && !log))
        return HBA_ERR_INVALID_ARGUMENT;
    if (h->policy != HBA_POLICY_SEGFIT) return HBA_ERR_INVALID_ARGUMENT;  // the loop runs segregated fit
    hba_serve_config_t c = cfg ? *cfg : hba_serve_config_t{};
    if (!c.queue_depth) c.queue_depth = 1u << 20;
    if (!c.max_batch) c.max_batch = 4096;
    if (!c.bucket_ns) c.bucket_ns = 262144;
    if (!c.time_limit_ns) c.time_limit_ns = 60ull * 1000000000ull;
    const uint32_t W = 4096, C = c.max_batch;
    hba::ServeArgs g{};
    g.ar = h->d_arenas;
    g.rec = h->d_rec;
    g.arr = reinterpret_cast<const hba::Arrival*>(arr);
    g.n = n;
    g.served = reinterpret_cast<hba::Served*>(served);
    g.log = log;
    g.log_cap = log_cap;
    g.qcap = c.queue_depth;
    g.W = W;
    g.C = C;
    g.bucket_ns = c.bucket_ns;
    g.max_batch = c.max_batch;
    g.time_limit_ns = c.time_limit_ns;
    g.max_ticks = c.max_ticks;
    if (h->serve_qcap < c.queue_depth || h->serve_batch < c.max_batch) {
        // first run, or one larger than any before: (re)allocate for the
        // largest queue and tick seen so far
        const uint32_t qcap = std::max(h->serve_qcap, c.queue_depth), bmax = std::max(h->serve_batch, c.max_batch);
        for (void*& p : h->serve_buf) {
            cudaFree(p);
            p = nullptr;
        }
        h->serve_qcap = h->serve_batch = 0;
        const size_t B = bmax;
        const size_t bytes[hba_s::SERVE_BUFS] = {4ull * qcap, 4ull * W * B, 4ull * W, 8 * B, 4 * B, 8 * B, 4 * B, 8 * B,
                                                 4 * hba::GATHER_WORDS * B, 4 * hba::SCRATCH_WORDS_PER_FREE * B,
                                                 sizeof(hba::ServeCtl)};
        for (int i = 0; i < hba_s::SERVE_BUFS; ++i) {
            if (cudaMalloc(&h->serve_buf[i], bytes[i]) != cudaSuccess) {
                (void)cudaGetLastError();
                for (void*& p : h->serve_buf) {
                    cudaFree(p);
                    p = nullptr;
                }
                return HBA_ERR_OUT_OF_MEMORY;
            }
        }
        h->serve_qcap = qcap;
        h->serve_batch = bmax;
    }
    g.queue = (uint32_t*)h->serve_buf[0];
    g.wheel = (uint32_t*)h->serve_buf[1];
    g.wheel_cnt = (uint32_t*)h->serve_buf[2];
    g.t_frees = (uint64_t*)h->serve_buf[3];
    g.t_fid = (uint32_t*)h->serve_buf[4];
    g.t_sizes = (uint64_t*)h->serve_buf[5];
    g.t_aid = (uint32_t*)h->serve_buf[6];
    g.t_out = (uint64_t*)h->serve_buf[7];
    g.gi = (uint32_t*)h->serve_buf[8];
    g.scr = (uint32_t*)h->serve_buf[9];
    g.ctl = (hba::ServeCtl*)h->serve_buf[10];
    hba_status_t r = HBA_OK;
    {
        static SmemLimits L{};
        static bool have = false;
        if (!have) {
            int dev = 0, optin = 48 * 1024;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, k_serve) == cudaSuccess) {
                L.single_dyn = (uint32_t)((optin - (int)fa.sharedSizeBytes - 1024) & ~15);
                cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.single_dyn);
            }
            have = true;
        }
        const uint32_t dyn = std::max<uint32_t>(L.single_dyn, 4 * hba::alloc_dyn_words<SERVE_NT>());
        if (cudaMemsetAsync(g.wheel_cnt, 0, 4ull * W, s) != cudaSuccess ||
            cudaMemsetAsync(g.ctl, 0, sizeof(hba::ServeCtl), s) != cudaSuccess ||
            (n && cudaMemsetAsync(served, 0, sizeof(hba_served_t) * n, s) != cudaSuccess))
            r = HBA_ERR_CUDA;
        if (r == HBA_OK) {
            k_serve<<<1, SERVE_NT, dyn, s>>>(g, dyn / 4);
            ++h->launches;
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) r = HBA_ERR_CUDA;
        }
        if (r == HBA_OK && cudaMemcpy(rep, g.ctl, sizeof(hba::ServeCtl), cudaMemcpyDeviceToHost) != cudaSuccess)
            r = HBA_ERR_CUDA;
        if (r == HBA_OK && rep->status == hba::SERVE_WHEEL_FULL) r = HBA_ERR_STATE;
    }
    return r;
}

// ---- batches that allocate nothing (hba_step_static) ----------------------
// Scratch for HBA_STATIC_MAX_FREES frees: the gathered records, then the
// free phase's global working arrays.  One array per device, shared by all
// calls; nothing in it needs clearing (a call writes every word it reads).
constexpr uint32_t STATIC_GI_WORDS = hba::GATHER_WORDS * HBA_STATIC_MAX_FREES;
constexpr uint32_t STATIC_WORDS = (hba::GATHER_WORDS + hba::SCRATCH_WORDS_PER_FREE) * HBA_STATIC_MAX_FREES;
static __device__ __align__(256) uint32_t g_static_scratch[STATIC_WORDS];

// Device address of g_static_scratch in the caller's current context, or
// nullptr on failure.  Host code cannot use the symbol's name as a device
// pointer, and the address differs between contexts: the module holding the
// array is loaded once per context, so after cudaDeviceReset, or under a
// context other than the device's primary one, the array lives elsewhere.
// The address is therefore looked up (cudaGetSymbolAddress, with the
// caller's context current) the first time each context calls, and kept
// under the context's unique id, which the driver never hands out twice in
// one process.  Without the driver's context calls it is looked up on every
// call.
using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);
std::mutex g_static_mu;
std::vector<std::pair<unsigned long long, uint32_t*>> g_static_addr;  // (context id, address)

bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        (void)cudaGetLastError();
    }
    if (!get_current || !get_id) return false;
    void* ctx = nullptr;
    return get_current(&ctx) == 0 && ctx && get_id(ctx, id) == 0;
}

uint32_t* static_scratch_address() {
    std::lock_guard<std::mutex> lock(g_static_mu);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (have_id)
        for (const auto& e : g_static_addr)
            if (e.first == id) return e.second;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    // the lookup makes the device's primary context current if none was
    if (have_id || current_context_id(&id)) g_static_addr.emplace_back(id, static_cast<uint32_t*>(p));
    return static_cast<uint32_t*>(p);
}

hba_status_t step_static_impl(hba_t h, const uint64_t* frees, uint32_t nf, uint8_t* st, const uint64_t* sizes,
                              uint32_t na, uint64_t* out, cudaStream_t s) {
    if (!h || h->n_arenas != 1) return HBA_ERR_INVALID_ARGUMENT;
    if ((nf && !frees) || (na && (!sizes || !out))) return HBA_ERR_INVALID_ARGUMENT;
    if (nf > HBA_STATIC_MAX_FREES) return HBA_ERR_INVALID_ARGUMENT;
    if (nf == 0 && na == 0) return HBA_OK;
    if (is_fit(h->policy)) return launch_fits(h, nullptr, frees, nf, st, nullptr, sizes, na, out, s);
    if (h->policy == HBA_POLICY_BITMASK) return launch_bitmask(h, nullptr, frees, nf, st, nullptr, sizes, na, out, s);
    uint32_t* base = static_scratch_address();
    if (!base) return HBA_ERR_CUDA;
    uint32_t* gi = base;
    uint32_t* scr = base + STATIC_GI_WORDS;
    return launch_single(h, frees, nf, st, sizes, na, out, s, gi, scr);
}

}  // namespace

extern "C" {

hba_status_t hba_serve_run(hba_t h, const hba_arrival_t* d_arrivals, uint64_t n, hba_served_t* d_served,
                           uint32_t* d_log, uint64_t log_cap, const hba_serve_config_t* cfg,
                           hba_serve_report_t* report, hba_stream_t stream) {
    StreamOrder order(h, (cudaStream_t)stream);
    return serve_impl(h, d_arrivals, n, d_served, d_log, log_cap, cfg, report, (cudaStream_t)stream);
}

hba_status_t hba_step_static(hba_t h, const uint64_t* d_frees, uint32_t nf, uint8_t* d_status,
                             const uint64_t* d_sizes, uint32_t na, uint64_t* d_out_offsets, hba_stream_t stream) {
    StreamOrder order(h, (cudaStream_t)stream);
    return step_static_impl(h, d_frees, nf, d_status, d_sizes, na, d_out_offsets, (cudaStream_t)stream);
}


const char* hba_version(void) { return "hba 0.1 (sm_103a)"; }

hba_status_t hba_launch_count(hba_t h, uint64_t* count) {
    if (!h || !count) return HBA_ERR_INVALID_ARGUMENT;
    *count = h->launches;
    return HBA_OK;
}

namespace {
// The per-arena lists of a TLSF handle and their initial state (one free
// block per arena).
// The per-arena structures of the policies other than segregated fit, and
// their initial state (one free block per arena).  The arena headers' bitmap
// field reports the first-level bitmap for TLSF, nothing for the fits.
hba_status_t alloc_policy(hba_t h, int policy) {
    h->policy = policy;
    const size_t n = h->h_init.size();
    if (policy == HBA_POLICY_TLSF) {
        h->h_tlsf.resize(n);
        for (size_t i = 0; i < n; ++i) {
            hba::tl_init_host(&h->h_tlsf[i], h->h_init[i].G);
            h->h_init[i].mask = h->h_tlsf[i].flmask;
        }
        if (cudaMalloc(&h->d_tlsf, sizeof(hba::TlsfLists) * n) != cudaSuccess) return HBA_ERR_OUT_OF_MEMORY;
    } else if (policy == HBA_POLICY_BITMASK) {
        h->h_bmh.resize(n);
        uint64_t words = 0;
        for (size_t i = 0; i < n; ++i) {
            const uint32_t W = (h->h_init[i].G + 63u) / 64u;
            if (W > hba::BM_MAX_WORDS) return HBA_ERR_INVALID_ARGUMENT;
            h->h_bmh[i] = hba::BmHdr{words, W, 0u};
            h->bm_wmax = std::max(h->bm_wmax, W);
            h->h_init[i].mask = 0;
            words += W;
        }
        if (cudaFuncSetAttribute(k_bitmask<BM_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(16u * hba::BM_MAX_WORDS)) != cudaSuccess)
            return HBA_ERR_CUDA;
        if (cudaMalloc(&h->d_bmh, sizeof(hba::BmHdr) * n) != cudaSuccess ||
            cudaMalloc(&h->d_bmF, 8 * words) != cudaSuccess || cudaMalloc(&h->d_bmS, 8 * words) != cudaSuccess)
            return HBA_ERR_OUT_OF_MEMORY;
    } else if (is_fit(policy)) {
        h->h_fhdr.assign(n, hba::FitHdr{1u, 0u, 0u, 0u});
        const uint32_t fit = policy == HBA_POLICY_FIRST_FIT ? hba::FIT_FIRST
                             : policy == HBA_POLICY_NEXT_FIT ? hba::FIT_NEXT : hba::FIT_BEST;
        for (size_t i = 0; i < n; ++i) {
            h->h_fhdr[i].fit = fit;
            h->h_init[i].mask = 0;
        }
        if (cudaFuncSetAttribute(k_fits<FIT_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(hba::FitBlk) * hba::FIT_RES)) != cudaSuccess)
            return HBA_ERR_CUDA;
        const size_t entries = h->total_granules + n;
        if (cudaMalloc(&h->d_fhdr, sizeof(hba::FitHdr) * n) != cudaSuccess ||
            cudaMalloc(&h->d_fpool, sizeof(hba::FitBlk) * entries) != cudaSuccess ||
            cudaMalloc(&h->d_upool, sizeof(hba::FitBlk) * entries) != cudaSuccess)
            return HBA_ERR_OUT_OF_MEMORY;
    }
    return HBA_OK;
}
bool known_policy(int policy) {
    return policy == HBA_POLICY_SEGFIT || policy == HBA_POLICY_TLSF || is_fit(policy) ||
           policy == HBA_POLICY_BITMASK;
}
}  // namespace

hba_status_t hba_create_ex(uint64_t arena_bytes, uint64_t min_block, int policy, uint32_t max_batch,
                           hba_t* out) {
    if (!out || !known_policy(policy) || max_batch == 0) return HBA_ERR_INVALID_ARGUMENT;
    uint32_t lg;
    uint64_t a;
    if (!check_geometry(arena_bytes, min_block, &lg, &a)) return HBA_ERR_INVALID_ARGUMENT;
    hba_t h = new hba_s();
    h->min_block = min_block;
    h->lg = lg;
    h->total_granules = a >> lg;
    h->max_batch = max_batch;
    std::vector<Arena> init(1);
    hba::arena_init_host(&init[0], a, lg, 0);
    hba_status_t r = alloc_meta(h, init, max_batch, max_batch);
    if (r == HBA_OK) r = alloc_policy(h, policy);
    if (r == HBA_OK) r = reset_impl(h, 0);
    if (r == HBA_OK && cudaDeviceSynchronize() != cudaSuccess) r = HBA_ERR_CUDA;
    if (r != HBA_OK) {
        free_all(h);
        delete h;
        return r;
    }
    *out = h;
    return HBA_OK;
}

hba_status_t hba_create(uint64_t arena_bytes, uint64_t min_block, int policy, hba_t* out) {
    return hba_create_ex(arena_bytes, min_block, policy, 65536, out);
}

hba_status_t hba_multi_create_ex(uint32_t n_arenas, const uint64_t* arena_bytes, uint64_t min_block, int policy,
                                 uint32_t max_total_frees, uint32_t max_total_allocs, hba_t* out) {
    if (!out || !arena_bytes || n_arenas == 0 || !known_policy(policy)) return HBA_ERR_INVALID_ARGUMENT;
    std::vector<Arena> init(n_arenas);
    uint64_t base = 0;
    uint32_t lg = 0;
    for (uint32_t i = 0; i < n_arenas; ++i) {
        uint64_t a;
        if (!check_geometry(arena_bytes[i], min_block, &lg, &a)) return HBA_ERR_INVALID_ARGUMENT;
        hba::arena_init_host(&init[i], a, lg, base);
        base += a >> lg;
    }
    hba_t h = new hba_s();
    h->min_block = min_block;
    h->lg = lg;
    h->total_granules = base;
    h->max_batch = max_total_frees;
    hba_status_t r = alloc_meta(h, init, max_total_frees, 0);
    if (r == HBA_OK && max_total_allocs) {
        r = make_pipeline(h, max_total_frees, max_total_allocs, (uint64_t)n_arenas + 1);
        h->stage_allocs = max_total_allocs;
    }
    if (r == HBA_OK) r = alloc_policy(h, policy);
    if (r == HBA_OK) r = reset_impl(h, 0);
    if (r == HBA_OK && cudaDeviceSynchronize() != cudaSuccess) r = HBA_ERR_CUDA;
    if (r != HBA_OK) {
        free_all(h);
        delete h;
        return r;
    }
    *out = h;
    return HBA_OK;
}

hba_status_t hba_multi_create(uint32_t n_arenas, const uint64_t* arena_bytes, uint64_t min_block, int policy,
                              uint32_t max_total_frees, hba_t* out) {
    return hba_multi_create_ex(n_arenas, arena_bytes, min_block, policy, max_total_frees, 0, out);
}

hba_status_t hba_destroy(hba_t h) {
    if (!h) return HBA_ERR_INVALID_ARGUMENT;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return HBA_OK;
}

hba_status_t hba_alloc_batch(hba_t h, const uint64_t* d_sizes, uint32_t n, uint64_t* d_out_offsets,
                             hba_stream_t stream) {
    StreamOrder order(h, (cudaStream_t)stream);
    return step_impl(h, nullptr, 0, nullptr, d_sizes, n, d_out_offsets, (cudaStream_t)stream);
}

hba_status_t hba_free_batch(hba_t h, const uint64_t* d_offsets, uint32_t n, hba_stream_t stream) {
    StreamOrder order(h, (cudaStream_t)stream);
    return step_impl(h, d_offsets, n, nullptr, nullptr, 0, nullptr, (cudaStream_t)stream);
}

hba_status_t hba_free_batch_ex(hba_t h, const uint64_t* d_offsets, uint32_t n, uint8_t* d_status,
                               hba_stream_t stream) {
    StreamOrder order(h, (cudaStream_t)stream);
    return step_impl(h, d_offsets, n, d_status, nullptr, 0, nullptr, (cudaStream_t)stream);
}

hba_status_t hba_step(hba_t h, const uint64_t* d_frees, uint32_t nf, uint8_t* d_status, const uint64_t* d_sizes,
                      uint32_t na, uint64_t* d_out_offsets, hba_stream_t stream) {
    StreamOrder order(h, (cudaStream_t)stream);
    return step_impl(h, d_frees, nf, d_status, d_sizes, na, d_out_offsets, (cudaStream_t)stream);
}

hba_status_t hba_step_host(hba_t h, const uint64_t* h_frees, uint32_t nf, uint8_t* h_status,
                           const uint64_t* h_sizes, uint32_t na, uint64_t* h_out_offsets, hba_stream_t stream) {
    if (!h || h->n_arenas != 1 || !h->d_stage_f) return HBA_ERR_INVALID_ARGUMENT;
    if (nf > h->max_batch || na > h->max_batch) return HBA_ERR_INVALID_ARGUMENT;
    if ((nf && !h_frees) || (na && (!h_sizes || !h_out_offsets))) return HBA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    StreamOrder order(h, s);
    if (nf) HBA_CUDA_TRY(cudaMemcpyAsync(h->d_stage_f, h_frees, 8ull * nf, cudaMemcpyHostToDevice, s));
    if (na) HBA_CUDA_TRY(cudaMemcpyAsync(h->d_stage_s, h_sizes, 8ull * na, cudaMemcpyHostToDevice, s));
    hba_status_t r = step_impl(h, h->d_stage_f, nf, h_status ? h->d_stage_st : nullptr, h->d_stage_s, na,
                               h->d_stage_o, s);
    if (r != HBA_OK) return r;
    if (na) HBA_CUDA_TRY(cudaMemcpyAsync(h_out_offsets, h->d_stage_o, 8ull * na, cudaMemcpyDeviceToHost, s));
    if (nf && h_status) HBA_CUDA_TRY(cudaMemcpyAsync(h_status, h->d_stage_st, nf, cudaMemcpyDeviceToHost, s));
    HBA_CUDA_TRY(cudaStreamSynchronize(s));
    return HBA_OK;
}

hba_status_t hba_step_host_async(hba_t h, const uint64_t* h_frees, uint32_t nf, uint8_t* h_status,
                                 const uint64_t* h_sizes, uint32_t na, uint64_t* h_out_offsets,
                                 hba_stream_t stream) {
    if (!h || h->n_arenas != 1 || !h->d_stage_f) return HBA_ERR_INVALID_ARGUMENT;
    if (nf > h->max_batch || na > h->max_batch) return HBA_ERR_INVALID_ARGUMENT;
    if ((nf && !h_frees) || (na && (!h_sizes || !h_out_offsets))) return HBA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HBA_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        // inside a capture every step stays on the captured stream, in order
        if (nf) HBA_CUDA_TRY(cudaMemcpyAsync(h->d_stage_f, h_frees, 8ull * nf, cudaMemcpyHostToDevice, s));
        if (na) HBA_CUDA_TRY(cudaMemcpyAsync(h->d_stage_s, h_sizes, 8ull * na, cudaMemcpyHostToDevice, s));
        hba_status_t r = step_impl(h, h->d_stage_f, nf, h_status ? h->d_stage_st : nullptr, h->d_stage_s, na,
                                   h->d_stage_o, s);
        if (r != HBA_OK) return r;
        if (na) HBA_CUDA_TRY(cudaMemcpyAsync(h_out_offsets, h->d_stage_o, 8ull * na, cudaMemcpyDeviceToHost, s));
        if (nf && h_status) HBA_CUDA_TRY(cudaMemcpyAsync(h_status, h->d_stage_st, nf, cudaMemcpyDeviceToHost, s));
        return HBA_OK;
    }
    hba_status_t r = HBA_OK;
    hba_s::Slot& q = h->slot[h->next_slot];
    h->next_slot ^= 1;
    // the slot's previous results must be out before its inputs are replaced
    if (q.used) HBA_CUDA_TRY(cudaStreamWaitEvent(h->s_in, q.out, 0));
    if (nf) HBA_CUDA_TRY(cudaMemcpyAsync(q.f, h_frees, 8ull * nf, cudaMemcpyHostToDevice, h->s_in));
    if (na) HBA_CUDA_TRY(cudaMemcpyAsync(q.s, h_sizes, 8ull * na, cudaMemcpyHostToDevice, h->s_in));
    HBA_CUDA_TRY(cudaEventRecord(q.in, h->s_in));
    HBA_CUDA_TRY(cudaStreamWaitEvent(h->s_run, q.in, 0));
    {
        StreamOrder order(h, h->s_run);
        r = step_impl(h, q.f, nf, h_status ? q.st : nullptr, q.s, na, q.o, h->s_run);
    }
    if (r != HBA_OK) return r;
    HBA_CUDA_TRY(cudaEventRecord(q.done, h->s_run));
    HBA_CUDA_TRY(cudaStreamWaitEvent(h->s_out, q.done, 0));
    if (na) HBA_CUDA_TRY(cudaMemcpyAsync(h_out_offsets, q.o, 8ull * na, cudaMemcpyDeviceToHost, h->s_out));
    if (nf && h_status) HBA_CUDA_TRY(cudaMemcpyAsync(h_status, q.st, nf, cudaMemcpyDeviceToHost, h->s_out));
    HBA_CUDA_TRY(cudaEventRecord(q.out, h->s_out));
    q.used = true;
    HBA_CUDA_TRY(cudaStreamWaitEvent(s, q.out, 0));
    return HBA_OK;
}

hba_status_t hba_reset(hba_t h, hba_stream_t stream) {
    if (!h) return HBA_ERR_INVALID_ARGUMENT;
    StreamOrder order(h, (cudaStream_t)stream);
    return reset_impl(h, (cudaStream_t)stream);
}

hba_status_t hba_stats(hba_t h, hba_stats_t* out) {
    if (!h || !out) return HBA_ERR_INVALID_ARGUMENT;
    HBA_CUDA_TRY(cudaDeviceSynchronize());
    if (h->d_fhdr) {  // the fits keep no record table: their lists give both figures
        k_fits_space<<<(h->n_arenas + 255) / 256, 256>>>(h->d_arenas, h->d_fhdr, h->d_fpool, h->d_upool,
                                                         h->n_arenas, h->d_largest, h->d_extent);
    } else if (h->d_bmh) {  // nor do the bitmask pools: their bitmaps do
        k_bm_space<<<(h->n_arenas + 255) / 256, 256>>>(h->d_arenas, h->d_bmh, h->d_bmF, h->d_bmS, h->n_arenas,
                                                       h->d_largest, h->d_extent);
    } else if (h->d_tlsf) {
        k_largest_tlsf<<<(h->n_arenas + 255) / 256, 256>>>(h->d_arenas, h->d_tlsf, h->d_rec, h->n_arenas,
                                                           h->d_largest);
    } else {
        k_largest<<<(h->n_arenas + 255) / 256, 256>>>(h->d_arenas, h->d_rec, h->n_arenas, h->d_largest);
    }
    ++h->launches;
    HBA_CUDA_TRY(cudaGetLastError());
    if (!h->d_fhdr && !h->d_bmh) {
        HBA_CUDA_TRY(cudaMemset(h->d_extent, 0, sizeof(uint32_t) * h->n_arenas));
        const uint64_t tiles = (h->total_granules + 64ull * 256 - 1) / (64ull * 256);
        const uint32_t grid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(tiles, 1), 8192);
        k_extent<<<grid, 256>>>(h->d_arenas, h->d_rec, h->n_arenas, h->total_granules, h->d_extent);
        ++h->launches;
        HBA_CUDA_TRY(cudaGetLastError());
    }
    std::vector<Arena> ar(h->n_arenas);
    std::vector<uint64_t> largest(h->n_arenas);
    std::vector<uint32_t> extent(h->n_arenas);
    HBA_CUDA_TRY(cudaMemcpy(ar.data(), h->d_arenas, sizeof(Arena) * h->n_arenas, cudaMemcpyDeviceToHost));
    HBA_CUDA_TRY(cudaMemcpy(largest.data(), h->d_largest, 8ull * h->n_arenas, cudaMemcpyDeviceToHost));
    HBA_CUDA_TRY(cudaMemcpy(extent.data(), h->d_extent, 4ull * h->n_arenas, cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->n_arenas = h->n_arenas;
    for (uint32_t i = 0; i < h->n_arenas; ++i) {
        const Arena& a = ar[i];
        out->alloc_ok += a.alloc_ok;
        out->alloc_fail += a.alloc_fail;
        out->free_ok += a.free_ok;
        out->free_fail += a.free_fail;
        out->used_bytes += (uint64_t)a.used_g << a.lg;
        out->used_blocks += a.used_blocks;
        out->blocks += a.blocks;
        out->requested_bytes += a.requested;
        out->arena_bytes += a.arena_bytes;
        out->largest_free = std::max(out->largest_free, largest[i]);
        out->extent_bytes += (uint64_t)extent[i] << a.lg;
        if (a.err && !out->device_error) out->device_error = a.err;
    }
    out->free_bytes = out->arena_bytes - out->used_bytes;
    out->bitmask = ar[0].mask << ar[0].lg;
    return out->device_error ? HBA_ERR_STATE : HBA_OK;
}

hba_status_t hba_export_state(hba_t h, uint32_t arena, uint64_t* host_buf, size_t cap, size_t* len) {
    if (!h || !len || arena >= h->n_arenas || (cap && !host_buf)) return HBA_ERR_INVALID_ARGUMENT;
    HBA_CUDA_TRY(cudaDeviceSynchronize());
    Arena ar;
    HBA_CUDA_TRY(cudaMemcpy(&ar, h->d_arenas + arena, sizeof(Arena), cudaMemcpyDeviceToHost));
    if (h->d_bmh) {
        hba::BmHdr H;
        HBA_CUDA_TRY(cudaMemcpy(&H, h->d_bmh + arena, sizeof(H), cudaMemcpyDeviceToHost));
        std::vector<uint64_t> F(H.words), S(H.words);
        HBA_CUDA_TRY(cudaMemcpy(F.data(), h->d_bmF + H.wbase, 8ull * H.words, cudaMemcpyDeviceToHost));
        HBA_CUDA_TRY(cudaMemcpy(S.data(), h->d_bmS + H.wbase, 8ull * H.words, cudaMemcpyDeviceToHost));
        *len = hba::bm_export(ar, H, F.data(), S.data(), host_buf, cap);
        return HBA_OK;
    }
    if (h->d_fhdr) {
        hba::FitHdr H;
        HBA_CUDA_TRY(cudaMemcpy(&H, h->d_fhdr + arena, sizeof(H), cudaMemcpyDeviceToHost));
        const uint64_t base = ar.rec_base + arena;
        std::vector<hba::FitBlk> fa(H.nfree), ua(H.nused);
        if (H.nfree)
            HBA_CUDA_TRY(cudaMemcpy(fa.data(), h->d_fpool + base, sizeof(hba::FitBlk) * H.nfree,
                                    cudaMemcpyDeviceToHost));
        if (H.nused)
            HBA_CUDA_TRY(cudaMemcpy(ua.data(), h->d_upool + base, sizeof(hba::FitBlk) * H.nused,
                                    cudaMemcpyDeviceToHost));
        *len = hba::fit_export(ar, H, fa.data(), ua.data(), host_buf, cap);
        return HBA_OK;
    }
    std::vector<Rec> rec(ar.G);
    HBA_CUDA_TRY(cudaMemcpy(rec.data(), h->d_rec + ar.rec_base, sizeof(Rec) * ar.G, cudaMemcpyDeviceToHost));
    if (h->d_tlsf) {
        hba::TlsfLists L;
        HBA_CUDA_TRY(cudaMemcpy(&L, h->d_tlsf + arena, sizeof(L), cudaMemcpyDeviceToHost));
        *len = hba::tl_export(ar, L, rec.data(), host_buf, cap);
        return HBA_OK;
    }
    *len = hba::export_canonical(ar, rec.data(), host_buf, cap);
    return HBA_OK;
}

hba_status_t hba_set_shape(hba_t h, uint32_t threads, uint32_t ctas, uint32_t smem_bytes) {
    if (!h) return HBA_ERR_INVALID_ARGUMENT;
    if (threads != 32 && threads != 64 && threads != 128 && threads != 256 && threads != 512 && threads != 1024)
        return HBA_ERR_INVALID_ARGUMENT;
    if (h->n_arenas == 1) {
        h->threads = threads;
        h->single_ctas = ctas;
    }
    h->m_threads = threads;
    h->m_ctas = ctas;
    h->smem_bytes = smem_bytes;
    return HBA_OK;
}

namespace {
hba_status_t multi_step_impl(hba_t h, const uint32_t* d_free_rowptr, const uint64_t* d_frees, uint32_t nf_total,
                             const uint32_t* d_alloc_rowptr, const uint64_t* d_sizes, uint32_t na_total,
                             uint64_t* d_out, uint8_t* d_free_status, cudaStream_t s) {
    const uint32_t n = h->n_arenas;
    const bool tl = h->policy == HBA_POLICY_TLSF;
    if (is_fit(h->policy))
        return launch_fits(h, d_free_rowptr, d_frees, nf_total, d_free_status, d_alloc_rowptr, d_sizes, na_total,
                           d_out, s);
    if (h->policy == HBA_POLICY_BITMASK)
        return launch_bitmask(h, d_free_rowptr, d_frees, nf_total, d_free_status, d_alloc_rowptr, d_sizes,
                              na_total, d_out, s);
    if (h->m_threads == 32) {
        // warp mode: WPC (WPC_TL) arenas per CTA, per-warp dynamic shared memory
        const SmemLimits& L = g_limits[5];
        const uint32_t aw = tl ? L.alloc_words_tl : L.alloc_words;
        const uint32_t wpc = tl ? WPC_TL : WPC;
        uint32_t per = std::min(h->smem_bytes ? h->smem_bytes : 4u * aw + 2048u, tl ? L.multi_dyn_tl : L.multi_dyn);
        per = (std::max(per, 4u * aw) + 15u) & ~15u;
        const uint32_t need = (n + wpc - 1) / wpc;
        const uint32_t grid = h->m_ctas ? std::min(h->m_ctas, need) : need;
        bool pdl = false;
        const bool pre = launch_prep(h, d_free_rowptr, d_frees, nf_total, h->d_gi, d_out, na_total, s, &pdl);
        if (cudaGetLastError() != cudaSuccess) return HBA_ERR_CUDA;
        const bool two = grid <= 2 * L.sms;
        cudaError_t e =
            tl ? launch_pdl(two ? k_multi_warp<2, 1, WPC_TL> : k_multi_warp<4, 1, WPC_TL>, grid, WPC_TL * 32,
                            per * WPC_TL, s, pdl, h->d_arenas, h->d_rec, d_free_rowptr, d_frees, d_free_status,
                            d_alloc_rowptr, d_sizes, d_out, h->d_scr, (const uint32_t*)h->d_gi, nf_total, n, per / 4,
                            pre ? 1u : 0u, h->d_tlsf)
               : launch_pdl(two ? k_multi_warp<2> : k_multi_warp<4>, grid, WPC * 32, per * WPC, s, pdl, h->d_arenas,
                            h->d_rec, d_free_rowptr, d_frees, d_free_status, d_alloc_rowptr, d_sizes, d_out, h->d_scr,
                            (const uint32_t*)h->d_gi, nf_total, n, per / 4, pre ? 1u : 0u, (hba::TlsfLists*)nullptr);
        if (e != cudaSuccess) return HBA_ERR_CUDA;
        ++h->launches;
        return cudaGetLastError() == cudaSuccess ? HBA_OK : HBA_ERR_CUDA;
    }
    const uint32_t grid = h->m_ctas ? std::min(h->m_ctas, n) : n;
    const int li = limit_index(h->m_threads);
    const uint32_t base = 4 * (tl ? g_limits[li].alloc_words_tl : g_limits[li].alloc_words);
    uint32_t dyn = std::min(h->smem_bytes ? h->smem_bytes : MULTI_DYN_BYTES_DEFAULT,
                            tl ? g_limits[li].multi_dyn_tl : g_limits[li].multi_dyn);
    dyn = (std::max(dyn, base) + 15u) & ~15u;
    const uint32_t dw = dyn / 4;
    bool pdl = false;
    const bool pre = launch_prep(h, d_free_rowptr, d_frees, nf_total, h->d_gi, d_out, na_total, s, &pdl);
    if (cudaGetLastError() != cudaSuccess) return HBA_ERR_CUDA;
    const uint32_t pf = pre ? 1u : 0u;
    Arena* ar = h->d_arenas;
    Rec* rec = h->d_rec;
    uint32_t* scr = h->d_scr;
    const uint32_t* gi = h->d_gi;
    cudaError_t e;
    hba::TlsfLists* lists = h->d_tlsf;
#define HBA_MULTI(NTV, POLV)                                                                                     \
    launch_pdl(k_multi<NTV, POLV>, grid, NTV, dyn, s, pdl, ar, rec, d_free_rowptr, d_frees, d_free_status,         \
               d_alloc_rowptr, d_sizes, d_out, scr, gi, nf_total, n, dw, pf, POLV ? lists : nullptr)
    switch (h->m_threads) {
        case 64: e = tl ? HBA_MULTI(64, 1) : HBA_MULTI(64, 0); break;
        case 128: e = tl ? HBA_MULTI(128, 1) : HBA_MULTI(128, 0); break;
        case 512: e = tl ? HBA_MULTI(512, 1) : HBA_MULTI(512, 0); break;
        case 1024: e = tl ? HBA_MULTI(1024, 1) : HBA_MULTI(1024, 0); break;
        default: e = tl ? HBA_MULTI(256, 1) : HBA_MULTI(256, 0); break;
    }
#undef HBA_MULTI
    if (e != cudaSuccess) return HBA_ERR_CUDA;
    ++h->launches;
    return cudaGetLastError() == cudaSuccess ? HBA_OK : HBA_ERR_CUDA;
}
}  // namespace

hba_status_t hba_multi_step(hba_t h, const uint32_t* d_free_rowptr, const uint64_t* d_frees, uint32_t nf_total,
                            const uint32_t* d_alloc_rowptr, const uint64_t* d_sizes, uint32_t na_total,
                            uint64_t* d_out, uint8_t* d_free_status, hba_stream_t stream) {
    if (!h || !d_free_rowptr || !d_alloc_rowptr) return HBA_ERR_INVALID_ARGUMENT;
    if (nf_total > h->scr_frees) return HBA_ERR_INVALID_ARGUMENT;
    if ((nf_total && !d_frees) || (na_total && (!d_sizes || !d_out))) return HBA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    StreamOrder order(h, s);
    return multi_step_impl(h, d_free_rowptr, d_frees, nf_total, d_alloc_rowptr, d_sizes, na_total, d_out,
                           d_free_status, s);
}

hba_status_t hba_multi_step_host_async(hba_t h, const uint32_t* h_free_rowptr, const uint64_t* h_frees,
                                       uint32_t nf_total, const uint32_t* h_alloc_rowptr, const uint64_t* h_sizes,
                                       uint32_t na_total, uint64_t* h_out, uint8_t* h_free_status,
                                       hba_stream_t stream) {
    if (!h || !h->stage_allocs || !h_free_rowptr || !h_alloc_rowptr) return HBA_ERR_INVALID_ARGUMENT;
    if (nf_total > h->scr_frees || na_total > h->stage_allocs) return HBA_ERR_INVALID_ARGUMENT;
    if ((nf_total && !h_frees) || (na_total && (!h_sizes || !h_out))) return HBA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rows = 4ull * ((size_t)h->n_arenas + 1);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HBA_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    const bool captured = cs != cudaStreamCaptureStatusNone;
    // inside a capture every step stays on the captured stream, in order,
    // through the first slot
    hba_s::Slot& q = h->slot[captured ? 0 : h->next_slot];
    cudaStream_t si = captured ? s : h->s_in, sr = captured ? s : h->s_run, so = captured ? s : h->s_out;
    if (!captured) {
        h->next_slot ^= 1;
        // the slot's previous results must be out before its inputs are replaced
        if (q.used) HBA_CUDA_TRY(cudaStreamWaitEvent(si, q.out, 0));
    }
    HBA_CUDA_TRY(cudaMemcpyAsync(q.fr, h_free_rowptr, rows, cudaMemcpyHostToDevice, si));
    HBA_CUDA_TRY(cudaMemcpyAsync(q.ar, h_alloc_rowptr, rows, cudaMemcpyHostToDevice, si));
    if (nf_total) HBA_CUDA_TRY(cudaMemcpyAsync(q.f, h_frees, 8ull * nf_total, cudaMemcpyHostToDevice, si));
    if (na_total) HBA_CUDA_TRY(cudaMemcpyAsync(q.s, h_sizes, 8ull * na_total, cudaMemcpyHostToDevice, si));
    if (!captured) {
        HBA_CUDA_TRY(cudaEventRecord(q.in, si));
        HBA_CUDA_TRY(cudaStreamWaitEvent(sr, q.in, 0));
    }
    hba_status_t r;
    {
        StreamOrder order(h, sr);
        r = multi_step_impl(h, q.fr, q.f, nf_total, q.ar, q.s, na_total, q.o, h_free_status ? q.st : nullptr, sr);
    }
    if (r != HBA_OK) return r;
    if (!captured) {
        HBA_CUDA_TRY(cudaEventRecord(q.done, sr));
        HBA_CUDA_TRY(cudaStreamWaitEvent(so, q.done, 0));
    }
    if (na_total) HBA_CUDA_TRY(cudaMemcpyAsync(h_out, q.o, 8ull * na_total, cudaMemcpyDeviceToHost, so));
    if (nf_total && h_free_status)
        HBA_CUDA_TRY(cudaMemcpyAsync(h_free_status, q.st, nf_total, cudaMemcpyDeviceToHost, so));
    if (!captured) {
        HBA_CUDA_TRY(cudaEventRecord(q.out, so));
        q.used = true;
        HBA_CUDA_TRY(cudaStreamWaitEvent(s, q.out, 0));
    }
    return HBA_OK;
}

}  // extern "C"
