// hba_engine.cuh -- per-arena batch engine of the header-free segregated-fit
// allocator (Bell, Kumar, Gill, arXiv 2405.07079, §5.1 Algorithms 4 and 5).
//
// One CTA applies one batch to one arena: every free in index order, then
// every allocation in index order, with results identical to the sequential
// algorithms.  The arena itself is never touched: the engine only reads and
// writes the out-of-band metadata below.
//
// Out-of-band metadata of one arena (the replacement for boundary tags, §3):
//   * a dense offset-to-block table, one 16-byte record per min_block granule
//     (a direct-indexed version of the address-keyed table of §3.3):
//        x = size in granules (bits 0..28) | state (bits 29..31)
//        y = granule of the previous adjacent block ("prev_adj", §3.3)
//        z = next block in its free list (free blocks; NIL for in-use ones)
//        w = previous block in its free list (free blocks)
//     Only records at block starts are meaningful; every other granule has
//     x == 0 (state NONE), which is what validates a free in O(1).
//   * per power-of-two class: the head of a doubly linked LIFO free list
//     (§5.1) and one bit of the availability bitmap (bit k <=> list k
//     non-empty).  Classes are counted in granules: class k holds blocks of
//     2^k .. 2^(k+1)-1 granules, i.e. byte class k + log2(min_block).
//
// How the sequential semantics is reached in parallel:
//   Free phase.  After validation (a free must name the start of an in-use
//   block; the lowest index wins among duplicates) the freed blocks form runs
//   of address-adjacent free blocks together with the free blocks they touch.
//   Applying the frees one by one leaves each run merged into one block whose
//   list push happened at the time of the LAST free inside the run (the last
//   free joins everything).  So: find each free's run (runs are disjoint
//   address ranges: with few runs, a search among the runs' leftmost frees;
//   otherwise pointer jumping over "predecessor freed block" links), take
//   per run the leftmost start, the right end and the largest free index,
//   unlink the absorbed free blocks, and push the merged blocks in
//   increasing order of that index.
//   Alloc phase.  Allocations only ever pop list heads and push remainders,
//   so the most recent remainder X is always the head of its list.  While
//   X's class L and the rest of the bitmap stay fixed, each request is
//   either a carve from X (lowest eligible list is L), a failure (no
//   eligible list), or an "other" pop from another list.  A block-wide scan
//   of carve sizes resolves a stretch of requests at once, up to the first
//   lane whose outcome differs from that speculation (an "other", or a carve
//   that X, shrunk by the carves before it, no longer serves); that event is
//   applied by one thread.  Where events are dense, one warp goes on with
//   warp-wide rounds (shuffles, no block barrier), or one thread applies the
//   next lanes one by one.  X's record is written ("materialised") only
//   when another remainder replaces it or the phase ends -- the
//   intermediate push/pop pairs of the sequential algorithm cancel out.
//
// Record reads for the frees are gathered before the engine runs, on many
// SMs (gather_free, one thread per free): one SM alone can keep only so many
// random loads in flight.  Small batches are gathered by the engine's own
// threads, four frees a thread at a time (gather_words4).
//
// The same source compiles for the GPU and, with HBA_EMULATE, for a
// host-only emulation used by the test suite: each HBA_FOR_THREADS body is a
// phase run by every thread, HBA_SYNC is the barrier between phases.  Inside
// a phase threads never read what another thread writes in that phase, except
// through atomics whose result is read after the barrier (and the pointer
// jumping, where any value read is a valid ancestor); warp-level exchanges
// (ballots, shuffles) have host versions written over the 32 lanes.
#pragma once
#include <type_traits>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#ifdef HBA_EMULATE
#include <string.h>
#define HBA_HD static inline
#define HBA_DEV static inline
#define HBA_FOR_THREADS(tid) for (int tid = 0; tid < NT; ++tid)
#define HBA_SYNC() \
    do {           \
    } while (0)
#define HBA_UNROLL
#else
#define HBA_UNROLL _Pragma("unroll")
#define HBA_HD __host__ __device__ __forceinline__
#define HBA_DEV __device__ __forceinline__
// NT == 32 is the warp mode: each warp of a CTA runs its own arena, the
// "barrier" is the warp's own __syncwarp and the thread index is the lane.
#define HBA_FOR_THREADS(tid) for (int tid = hba_tid<NT, POL>(); tid < NT; tid += NT)
#define HBA_SYNC() hba_sync<NT, POL>()
template <int NT, int POL = 0>
__device__ __forceinline__ int hba_tid() {
    return NT == 32 ? (int)(threadIdx.x & 31u) : (int)threadIdx.x;
}
template <int NT, int POL = 0>
__device__ __forceinline__ void hba_sync() {
    if (NT == 32) __syncwarp();
    else __syncthreads();
}
#endif

// Phase-boundary hook for timing probes; compiled out unless a probe build
// defines it.
#ifndef HBA_PROF
#define HBA_PROF(slot) \
    do {               \
    } while (0)
#endif

namespace hba {

constexpr uint32_t NIL = 0xFFFFFFFFu;
constexpr uint32_t SZ_BITS = 29;
constexpr uint32_t SZ_MASK = (1u << SZ_BITS) - 1u;
constexpr uint32_t MAX_GRANULES = SZ_MASK;  // G <= 2^29 - 1
constexpr uint32_t ST_NONE = 0, ST_USED = 1, ST_FREE = 2, ST_NEW = 3, ST_DEL = 4;
constexpr uint64_t FAIL64 = ~0ull;
constexpr int NBINS = 32;  // granule classes 0..28 are reachable
// global scratch per free: absorbed blocks (2 words) always; the free
// phase's working arrays (table < 8, 7 per-free arrays, 2 absorbed) when
// they do not fit in shared memory
constexpr uint32_t SCRATCH_WORDS_PER_FREE = 18;
constexpr uint32_t GATHER_WORDS = 5;
// alloc phase: after a block-wide round that resolved fewer than
// STRETCH_BELOW lanes before its event, one warp goes on through up to
// STRETCH_LANES lanes with warp-wide rounds (no block barrier), until a
// window of 32 lanes holds no event
#ifndef HBA_STRETCH_BELOW
#define HBA_STRETCH_BELOW 256
#endif
#ifndef HBA_STRETCH_LANES
#define HBA_STRETCH_LANES 512
#endif
// Where events come one after another (the event is the first unresolved
// lane), speculation resolves nothing: one thread applies the next
// SERIAL_LANES lanes one by one instead.
#ifndef HBA_SERIAL_LANES
#define HBA_SERIAL_LANES 64
#endif
constexpr uint32_t STRETCH_BELOW = HBA_STRETCH_BELOW;
constexpr uint32_t STRETCH_LANES = HBA_STRETCH_LANES;
constexpr uint32_t SERIAL_LANES = HBA_SERIAL_LANES;
#ifndef HBA_QUIET_RUN
#define HBA_QUIET_RUN 4
#endif
constexpr uint32_t QUIET_RUN = HBA_QUIET_RUN;
// ... and at most QUIET_FIRST such lanes before the run's first further pop
#ifndef HBA_QUIET_FIRST
#define HBA_QUIET_FIRST 0
#endif
constexpr uint32_t QUIET_FIRST = HBA_QUIET_FIRST;
// a block-wide round that resolved at most SERIAL_AFTER lanes before its
// event counts as "events one after another"
#ifndef HBA_SERIAL_AFTER
#define HBA_SERIAL_AFTER 2
#endif
constexpr uint32_t SERIAL_AFTER = HBA_SERIAL_AFTER;
// record tables up to this size are prefetched into L2 whole at batch start
#ifndef HBA_PREFETCH_TABLE_MAX
#define HBA_PREFETCH_TABLE_MAX (2u << 20)
#endif
constexpr uint64_t PREFETCH_TABLE_MAX = HBA_PREFETCH_TABLE_MAX;
// free phase: with at most LEAD_MAX runs, every free finds its run by a
// search among the runs' leaders (in address order); otherwise by pointer
// jumping, following JUMP_HOPS links per pass.  With at most SERIAL_PUSH_MAX
// runs, one thread pushes the merged blocks; otherwise segments of the push
// order are linked in parallel.
#ifndef HBA_LEAD_MAX
#define HBA_LEAD_MAX 64
#endif
#ifndef HBA_SERIAL_PUSH_MAX
#define HBA_SERIAL_PUSH_MAX 8
#endif
constexpr uint32_t LEAD_MAX = HBA_LEAD_MAX;
// free batches up to this size stage their gathered records in shared memory
#ifndef HBA_STAGE_MAX_FREES
#define HBA_STAGE_MAX_FREES 1024
#endif
constexpr uint32_t STAGE_MAX_FREES = HBA_STAGE_MAX_FREES;
constexpr uint32_t SERIAL_PUSH_MAX = HBA_SERIAL_PUSH_MAX;
static_assert(SERIAL_PUSH_MAX <= LEAD_MAX, "the serial push uses the leader search's order");
constexpr int JUMP_HOPS = 2;
// device error codes (Arena::err); any of them means corrupted metadata
constexpr uint32_t ERR_LIST_WALK = 1;   // an unlink walk ran past the block count
constexpr uint32_t ERR_EMPTY_HEAD = 2;  // a class with its bit set had no head

struct alignas(16) Rec {
    uint32_t x, y, z, w;
};

// Per-arena header, resident in device memory between batches.
struct Arena {
    uint64_t arena_bytes;  // managed bytes, a multiple of min_block
    uint64_t rec_base;     // index of the arena's first record in the record pool
    uint32_t G;            // granules
    uint32_t lg;           // log2(min_block)
    uint32_t heads[NBINS]; // list heads per granule class, NIL if empty
    uint64_t mask;         // availability bitmap over granule classes
    int64_t alloc_ok, alloc_fail, free_ok, free_fail;
    int64_t used_g, used_blocks, blocks, requested;
    uint32_t err, pad;
};

HBA_HD uint32_t st_of(uint32_t x) { return x >> SZ_BITS; }
HBA_HD uint32_t sz_of(uint32_t x) { return x & SZ_MASK; }
HBA_HD uint32_t mkx(uint32_t sz, uint32_t st) { return sz | (st << SZ_BITS); }

#ifdef HBA_EMULATE
HBA_HD uint32_t flog2(uint32_t v) { return 31u - (uint32_t)__builtin_clz(v); }
HBA_HD uint32_t ctz64(uint64_t v) { return (uint32_t)__builtin_ctzll(v); }
#else
HBA_HD uint32_t flog2(uint32_t v) {
#ifdef __CUDA_ARCH__
    return 31u - (uint32_t)__clz(v);
#else
    return 31u - (uint32_t)__builtin_clz(v);
#endif
}
HBA_HD uint32_t ctz64(uint64_t v) {
#ifdef __CUDA_ARCH__
    return (uint32_t)(__ffsll((long long)v) - 1);
#else
    return (uint32_t)__builtin_ctzll(v);
#endif
}
#endif
// ceil(log2 v) for v >= 1
HBA_HD uint32_t clog2(uint32_t v) { return v <= 1 ? 0u : flog2(v - 1) + 1u; }

// ---- two-level segregated fit (§5.2): lists and their arithmetic ---------
// Sizes in granules.  With 16 lists per class (the paper gives no count),
// the list of a free block of r granules is (f, s): f = floor(log2 r) and s
// the four bits below the leading one, so list (f, s) holds the sizes
// [2^f + s 2^f / 16, 2^f + (s + 1) 2^f / 16); its index is 16 f + s.
constexpr uint32_t TL_SLB = 4;                 // log2 of the lists per class
constexpr uint32_t TL_SL = 1u << TL_SLB;       // 16
constexpr uint32_t TL_FL = 32;                 // granule classes (G < 2^29)
constexpr uint32_t TL_NL = TL_FL * TL_SL;      // 512 lists
constexpr uint32_t TL_NONE = 0xFFFFFFFFu;

static_assert(TL_FL == 32, "one second-level mask per lane of a warp");

struct TlsfLists {
    uint32_t flmask;           // bit f <=> slmask[f] != 0
    uint32_t pad;
    uint16_t slmask[TL_FL];    // bit s of slmask[f] <=> list (f, s) non-empty
    uint32_t heads[TL_NL];     // list f * 16 + s: first block (granule), NIL if empty
};

// List of a free block of r >= 1 granules.
HBA_HD uint32_t tl_list(uint32_t r) {
    const uint32_t f = flog2(r);
    const uint32_t top = f >= TL_SLB ? r >> (f - TL_SLB) : r << (TL_SLB - f);  // 16 + s
    return f * TL_SL + (top - TL_SL);
}

// Lowest list whose lower bound is >= r: r rounded up to a list bound.
HBA_HD uint32_t tl_bound(uint32_t r) {
    const uint32_t f = flog2(r);
    const uint32_t up = f >= TL_SLB ? r + ((1u << (f - TL_SLB)) - 1u) : r;  // r < 2^29: no overflow
    return tl_list(up);
}


// ---- memory helpers ------------------------------------------------------
#ifdef HBA_EMULATE
HBA_DEV Rec ldr(const Rec* r, uint32_t g) { return r[g]; }
HBA_DEV void str(Rec* r, uint32_t g, Rec v) { r[g] = v; }
HBA_DEV uint32_t at_min_u32(uint32_t* p, uint32_t v) { uint32_t o = *p; if (v < o) *p = v; return o; }
HBA_DEV uint32_t at_max_u32(uint32_t* p, uint32_t v) { uint32_t o = *p; if (v > o) *p = v; return o; }
HBA_DEV uint32_t at_add_u32(uint32_t* p, uint32_t v) { uint32_t o = *p; *p = o + v; return o; }
HBA_DEV void at_add_i64(int64_t* p, int64_t v) { *p += v; }
HBA_DEV uint32_t at_cas_u32(uint32_t* p, uint32_t cmp, uint32_t v) { uint32_t o = *p; if (o == cmp) *p = v; return o; }
HBA_DEV uint64_t at_cas_u64(uint64_t* p, uint64_t cmp, uint64_t v) { uint64_t o = *p; if (o == cmp) *p = v; return o; }
HBA_DEV uint64_t at_min_u64(uint64_t* p, uint64_t v) { uint64_t o = *p; if (v < o) *p = v; return o; }
#else
HBA_DEV Rec ldr(const Rec* r, uint32_t g) {
    uint4 v = *reinterpret_cast<const uint4*>(r + g);
    return Rec{v.x, v.y, v.z, v.w};
}
HBA_DEV void str(Rec* r, uint32_t g, Rec v) { *reinterpret_cast<uint4*>(r + g) = make_uint4(v.x, v.y, v.z, v.w); }
HBA_DEV uint32_t at_min_u32(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
HBA_DEV uint32_t at_max_u32(uint32_t* p, uint32_t v) { return atomicMax(p, v); }
HBA_DEV uint32_t at_add_u32(uint32_t* p, uint32_t v) { return atomicAdd(p, v); }
HBA_DEV uint32_t at_cas_u32(uint32_t* p, uint32_t cmp, uint32_t v) { return atomicCAS(p, cmp, v); }
HBA_DEV uint64_t at_cas_u64(uint64_t* p, uint64_t cmp, uint64_t v) {
    return atomicCAS(reinterpret_cast<unsigned long long*>(p), (unsigned long long)cmp, (unsigned long long)v);
}
HBA_DEV uint64_t at_min_u64(uint64_t* p, uint64_t v) {
    return atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
HBA_DEV void at_add_i64(int64_t* p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
#endif

// ---- gathering the records a free needs (one thread per free) ------------
// For a free of byte offset `off`: the block it names (if it is the start of
// an in-use block), and the two address neighbours' facts that coalescing
// needs.  Written as five words per free (structure of arrays, stride n):
//   g     the block's first granule, NIL if the free is not valid
//   szf   its size in granules | Lfree << 29 | Rfree << 30
//   L     its left neighbour (prev_adj), NIL at offset 0
//   LL    the left neighbour's own left neighbour when the left one is free
//   Rend  end of the right neighbour when that one is free, else end of the block
constexpr uint32_t F_LFREE = 1u << 29, F_RFREE = 1u << 30;
HBA_HD void gather_words(const Rec* rec, uint64_t A, uint32_t G, uint32_t lg, uint64_t off,
                         uint32_t w[GATHER_WORDS]) {
    uint32_t g = NIL, szf = 0, L = NIL, LL = NIL, Rend = 0;
    if (off < A && (off & ((1ull << lg) - 1ull)) == 0) {
        const uint32_t gg = (uint32_t)(off >> lg);
        const Rec r = rec[gg];
        if (st_of(r.x) == ST_USED) {
            g = gg;
            const uint32_t sz = sz_of(r.x);
            szf = sz;
            L = r.y;
            Rend = gg + sz;
            // both neighbours are independent loads
            const Rec rl = L != NIL ? rec[L] : Rec{0, NIL, 0, 0};
            const uint32_t rx = Rend < G ? rec[Rend].x : 0u;
            if (st_of(rl.x) == ST_FREE) {
                szf |= F_LFREE;
                LL = rl.y;
            }
            if (st_of(rx) == ST_FREE) {
                szf |= F_RFREE;
                Rend += sz_of(rx);
            }
        }
    }
    w[0] = g;
    w[1] = szf;
    w[2] = L;
    w[3] = LL;
    w[4] = Rend;
}
// The same for up to four frees at once, their record loads issued side by
// side (first the named blocks, then all their neighbours): one thread keeps
// several independent loads in flight.  valid[e] false: w[e] is not written.
HBA_HD void gather_words4(const Rec* rec, uint64_t A, uint32_t G, uint32_t lg, const uint64_t off[4],
                          const bool valid[4], uint32_t w[4][GATHER_WORDS]) {
    uint32_t gg[4];
    Rec r[4];
    HBA_UNROLL
    for (int e = 0; e < 4; ++e) {
        gg[e] = NIL;
        r[e] = Rec{0, NIL, 0, 0};
        if (valid[e] && off[e] < A && (off[e] & ((1ull << lg) - 1ull)) == 0) {
            gg[e] = (uint32_t)(off[e] >> lg);
            r[e] = rec[gg[e]];
        }
    }
    Rec rl[4];
    uint32_t rx[4];
    HBA_UNROLL
    for (int e = 0; e < 4; ++e) {
        rl[e] = Rec{0, NIL, 0, 0};
        rx[e] = 0;
        if (gg[e] != NIL && st_of(r[e].x) == ST_USED) {
            const uint32_t L = r[e].y, Rend = gg[e] + sz_of(r[e].x);
            if (L != NIL) rl[e] = rec[L];
            if (Rend < G) rx[e] = rec[Rend].x;
        }
    }
    HBA_UNROLL
    for (int e = 0; e < 4; ++e) {
        if (!valid[e]) continue;
        uint32_t g = NIL, szf = 0, L = NIL, LL = NIL, Rend = 0;
        if (gg[e] != NIL && st_of(r[e].x) == ST_USED) {
            g = gg[e];
            const uint32_t sz = sz_of(r[e].x);
            szf = sz;
            L = r[e].y;
            Rend = g + sz;
            if (st_of(rl[e].x) == ST_FREE) {
                szf |= F_LFREE;
                LL = rl[e].y;
            }
            if (st_of(rx[e]) == ST_FREE) {
                szf |= F_RFREE;
                Rend += sz_of(rx[e]);
            }
        }
        w[e][0] = g;
        w[e][1] = szf;
        w[e][2] = L;
        w[e][3] = LL;
        w[e][4] = Rend;
    }
}
HBA_HD void gather_free(const Rec* rec, uint64_t A, uint32_t G, uint32_t lg, uint64_t off, uint32_t* gi,
                        uint32_t n, uint32_t j) {
    uint32_t w[GATHER_WORDS];
    gather_words(rec, A, G, lg, off, w);
    for (uint32_t q = 0; q < GATHER_WORDS; ++q) gi[q * n + j] = w[q];
}

// ---- shared state of one CTA --------------------------------------------
enum : uint8_t { CL_NONE = 0, CL_FAIL = 1, CL_CARVE = 2, CL_OTHER = 3 };
// counter slots (per warp, plus one row for single-thread updates)
enum : int { C_AOK = 0, C_AFAIL, C_FOK, C_FFAIL, C_USEDG, C_REQ, C_NOSPLIT, C_BLOCKS, NCNT };

// POL selects the class layout of the free lists: 0, segregated fit (§5.1:
// 32 classes, a block of r granules in class floor(log2 r), one bitmap
// word); 1, two-level segregated fit (§5.2: the 512 lists above, the first
// level in the bitmap word, the second level per class in tsl).
template <int NT, int POL = 0>
struct Smem {
    static constexpr int NW = NT >= 32 ? NT / 32 : 1;
    static constexpr int NSEG = NT >= 16 ? NT / 16 : 1;  // segments of the push order
    static constexpr int NCLS = POL ? (int)TL_NL : NBINS;
    using ccl_t = typename std::conditional<POL == 0, uint8_t, uint16_t>::type;
    uint64_t A;          // arena bytes
    uint64_t mask;       // bitmap of classes (POL 1: first level) whose list is non-empty (X excluded)
    uint32_t heads[NCLS];
    uint32_t G, lg;
    // the most recent remainder X: virtual head of class xL while xok
    uint32_t xok, xg, xsz, xright, xL, xprev;
    uint32_t c0g, c0sz, c0prev;  // X when the current round classified its lanes
    Rec hc[NCLS];        // record of each list head (alloc phase), refilled asynchronously
    // loop control
    uint32_t p, r, cont, evb[2], nul, nruns, flag[3];
    // free phase: run leaders (applied frees with nothing applied to their
    // left in the run) in address order, when there are at most LEAD_MAX
    uint32_t nlead, lead[LEAD_MAX], lkey[LEAD_MAX], lsort[LEAD_MAX];
    uint32_t err;        // first metadata error seen by this CTA (0 = none)
    uint32_t* dyn;       // dynamic shared memory
    uint32_t dyn_words;
    // alloc-phase arrays (carved from dyn)
    int64_t* val;        // carve sizes, then their inclusive prefix
    uint64_t* s64;       // request sizes of the chunk
    uint64_t* stg;       // [2][NT] request sizes of the next chunk, copied in ahead
    uint32_t* cst;       // start granule of each carve lane
    uint32_t* sgr;       // rounded sizes in granules (0: invalid request)
    uint8_t* cls;        // class of each lane in the current round
    ccl_t* ccl;          // size class c (the threshold class) of each lane
    int64_t wc[NW + 1][NCNT];
    int64_t warp_tot[32];
    uint32_t wlast[32];  // start of the highest carve lane of each warp (NIL: none)
    uint32_t wcm[32];    // carve lanes of each warp in the current round
    uint32_t segf[NSEG][POL ? 1 : NBINS];  // oldest run of each class per push segment (POL 0)
    uint32_t segl[NSEG][POL ? 1 : NBINS];  // newest run of each class per push segment (POL 0)
    uint32_t cnt[NT];
    uint32_t tsl[POL ? TL_FL : 1];  // POL 1: second-level bitmap of each first-level class
};

// words of dynamic shared memory the alloc phase carves for NT lanes
template <int NT, int POL = 0>
HBA_HD uint32_t alloc_dyn_words() { return 2 * NT + 2 * NT + 4 * NT + NT + NT + NT / 4 + (POL ? NT / 2 : NT / 4) + 8; }

// ---- the class layout (POL) ---------------------------------------------
constexpr uint32_t CLS_NONE = 0xFFFFFFFFu;
// class of a free block of r granules
template <int POL>
HBA_HD uint32_t cls_push(uint32_t r) { return POL ? tl_list(r) : flog2(r); }
// lowest class whose every block fits a request of sg granules
template <int POL>
HBA_HD uint32_t cls_req(uint32_t sg) { return POL ? tl_bound(sg) : clog2(sg); }
// Lowest non-empty class at or above t, with class xl counted non-empty
// when xok (the virtual remainder X); CLS_NONE if none.  mask: the bitmap
// word (POL 1: the first level; the second level is S.tsl).  The hot sites
// spell out the POL 0 case as a candidate mask ((bitmap >> t) << t, lowest
// set bit), which compiles to shorter dependent chains there than going
// through this function (measured: 4 % on the batched form).
template <int NT, int POL>
HBA_HD uint32_t cls_first(const Smem<NT, POL>& S, uint64_t mask, uint32_t t, bool xok, uint32_t xl) {
    if constexpr (POL == 0) {
        const uint64_t cand = ((mask | (xok ? (1ull << xl) : 0ull)) >> t) << t;
        return cand ? ctz64(cand) : CLS_NONE;
    } else {
        const uint32_t f = t >> TL_SLB, sb = t & (TL_SL - 1);
        const uint32_t xf = xl >> TL_SLB, xb = 1u << (xl & (TL_SL - 1));
        uint32_t here = S.tsl[f] | (xok && xf == f ? xb : 0u);
        here &= 0xFFFFu << sb;
        if (here) return (f << TL_SLB) + ctz64(here);
        uint64_t fl = mask | (xok ? (1ull << xf) : 0ull);
        fl = (fl >> (f + 1)) << (f + 1);
        if (!fl) return CLS_NONE;
        const uint32_t f2 = ctz64(fl);
        const uint32_t sl = S.tsl[f2] | (xok && xf == f2 ? xb : 0u);
        return (f2 << TL_SLB) + ctz64(sl);
    }
}
// Mark class k non-empty or empty (one thread).
template <int NT, int POL>
HBA_HD void cls_mark(Smem<NT, POL>& S, uint64_t& mask, uint32_t k, bool nonempty) {
    if constexpr (POL == 0) {
        if (nonempty) mask |= 1ull << k;
        else mask &= ~(1ull << k);
    } else {
        const uint32_t f = k >> TL_SLB, b = 1u << (k & (TL_SL - 1));
        const uint32_t sl = nonempty ? (S.tsl[f] | b) : (S.tsl[f] & ~b);
        S.tsl[f] = sl;
        if (sl) mask |= 1ull << f;
        else mask &= ~(1ull << f);
    }
}

// ---- warp-aggregated counters and votes (call convergently) --------------
template <int NT, int POL = 0>
HBA_DEV void warp_count(Smem<NT, POL>& S, int tid, int k, bool pred) {
#ifdef HBA_EMULATE
    S.wc[tid / 32][k] += pred ? 1 : 0;
#else
    const unsigned b = __ballot_sync(0xffffffffu, pred);
    if ((tid & 31) == 0) S.wc[tid >> 5][k] += __popc(b);
#endif
}
template <int NT, int POL = 0>
HBA_DEV void warp_sum(Smem<NT, POL>& S, int tid, int k, int64_t v) {
#ifdef HBA_EMULATE
    S.wc[tid / 32][k] += v;
#else
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) S.wc[tid >> 5][k] += v;
#endif
}
// single-thread counter update (its own row: never races with warp_*)
template <int NT, int POL = 0>
HBA_DEV void single_add(Smem<NT, POL>& S, int k, int64_t v) { S.wc[Smem<NT, POL>::NW][k] += v; }

HBA_DEV void prefetch_l2(const void* p) {
#ifdef HBA_EMULATE
    (void)p;
#else
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
#endif
}

// Asynchronous copies into shared memory (a 16-byte record, an 8-byte request
// size), and the wait for all of the calling thread's outstanding copies.
HBA_DEV void rec_copy_async(Rec* dst_smem, const Rec* src) {
#ifdef HBA_EMULATE
    *dst_smem = *src;
#else
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
#endif
}
HBA_DEV void u64_copy_async(uint64_t* dst_smem, const uint64_t* src) {
#ifdef HBA_EMULATE
    *dst_smem = *src;
#else
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
#endif
}
HBA_DEV void rec_copy_wait() {
#ifndef HBA_EMULATE
    asm volatile("cp.async.wait_all;" ::: "memory");
#endif
}

// ---- block-wide collectives (called by all threads, outside phases) ------
// Inclusive prefix sum over the lanes of the warps that intersect the lane
// window [lo, hi): thread tid of such a warp gets its inclusive prefix back
// (also stored in v[tid]); warps outside the window contribute nothing, do
// no shuffles and leave their v[] untouched.  One barrier inside; on return
// only the caller's own v[tid] may be read without another barrier.
template <int NT, int POL = 0>
HBA_DEV bool warp_in_window(int wid, uint32_t lo, uint32_t hi) {
    const uint32_t w0 = (uint32_t)wid * 32u, w1 = w0 + 32u;
    return w0 < hi && lo < w1;
}
template <int NT, int POL = 0>
HBA_DEV int64_t scan_incl_i64(Smem<NT, POL>& S, int64_t* v, uint32_t lo, uint32_t hi) {
#ifdef HBA_EMULATE
    int64_t run = 0;
    for (int i = 0; i < NT; ++i)
        if (warp_in_window<NT, POL>(i / 32, lo, hi)) {
            run += v[i];
            v[i] = run;
        }
    (void)S;
    return 0;
#else
    const int tid = hba_tid<NT, POL>(), lane = tid & 31, wid = tid >> 5;
    const bool act = warp_in_window<NT, POL>(wid, lo, hi);
    int64_t x = act ? v[tid] : 0;
    if (act) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
    }
    if (NT == 32) {
        __syncwarp();
    } else {
        if (lane == 31) S.warp_tot[wid] = x;
        __syncthreads();
        if (act) {
            // every active warp sums the totals of the warps below it itself:
            // no second barrier
            const int w0 = (int)(lo >> 5);
            int64_t t = lane >= w0 && lane < wid ? S.warp_tot[lane] : 0;
#pragma unroll
            for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            x += t;
        }
    }
    if (act) v[tid] = x;
    return x;
#endif
}

// Exclusive prefix sum of c[0..NT) in place; *total receives the sum.
// Followed by a barrier.
template <int NT, int POL = 0>
HBA_DEV void scan_excl_u32(Smem<NT, POL>& S, uint32_t* c, uint32_t* total) {
#ifdef HBA_EMULATE
    uint32_t run = 0;
    for (int i = 0; i < NT; ++i) {
        uint32_t t = c[i];
        c[i] = run;
        run += t;
    }
    *total = run;
    (void)S;
#else
    const int tid = hba_tid<NT, POL>(), lane = tid & 31, wid = tid >> 5;
    int64_t own = c[tid];
    int64_t x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (NT > 32) {
        if (lane == 31) S.warp_tot[wid] = x;
        __syncthreads();
        int64_t t = lane < NT / 32 ? S.warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        const int64_t before = __shfl_sync(0xffffffffu, t, (wid + 31) & 31);
        if (wid > 0) x += before;
    }
    c[tid] = (uint32_t)(x - own);
    if (tid == NT - 1) *total = (uint32_t)x;
    hba_sync<NT, POL>();
#endif
}

struct StepArgs {
    Arena* ar;
    Rec* rec;        // the arena's records (already offset by rec_base)
    const uint64_t* frees;
    uint32_t nf;
    uint8_t* fstat;  // may be null
    const uint64_t* sizes;
    uint32_t na;
    uint64_t* out;
    uint32_t* scr;   // SCRATCH_WORDS_PER_FREE * nf words of global scratch
    const uint32_t* gi;  // gathered records of the frees (5 arrays of stride gstride)
    uint32_t gstride;
    uint32_t prefilled;  // out[] already holds HBA_FAIL everywhere (written by a
                         // preceding grid): failures need no store
    uint32_t wait_prep;  // after reading the arena header, before touching what
                         // the gathering threads write (gathered records, out[]):
                         // WAIT_NONE, WAIT_GRID (preceding grid, programmatic
                         // dependent launch) or WAIT_CLUSTER (the other CTAs of
                         // this cluster)
    uint32_t staged;     // the gathered records are already in the free phase's
                         // shared-memory layout (written there by the cluster)
    uint32_t self_gather;  // no gathering grid ran: the CTA gathers its frees'
                           // records itself (small batches), into the free
                           // phase's shared-memory layout or, when that does
                           // not fit, into gi
    TlsfLists* tl;         // two-level segregated fit (POL 1): the arena's list heads and bitmaps
};
constexpr uint32_t WAIT_NONE = 0, WAIT_GRID = 1, WAIT_CLUSTER = 2;

HBA_DEV void grid_dep_wait() {
#ifndef HBA_EMULATE
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
// Cluster barrier halves: the engine CTA arrives early (it publishes nothing)
// and waits when it needs what the other CTAs wrote; they arrive with release
// semantics once their writes are done.
HBA_DEV void cluster_arrive_relaxed() {
#ifndef HBA_EMULATE
    asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
#endif
}
HBA_DEV void cluster_arrive_release() {
#ifndef HBA_EMULATE
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
#endif
}
HBA_DEV void cluster_wait() {
#ifndef HBA_EMULATE
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
#endif
}

// The virtual remainder X, the bitmap and the counters of the one thread that
// applies requests one by one, held in registers while it does (loaded from
// and stored back to shared memory around each serial stretch).
struct XReg {
    uint64_t mask;
    uint32_t xok, xg, xsz, xL, xprev, xright, lg, G;
    int64_t aok, afail, usedg, req, nosplit;
};
template <int NT, int POL = 0>
HBA_DEV XReg x_load(const Smem<NT, POL>& S) {
    return XReg{S.mask, S.xok, S.xg, S.xsz, S.xL, S.xprev, S.xright, S.lg, S.G, 0, 0, 0, 0, 0};
}
template <int NT, int POL = 0>
HBA_DEV void x_store(Smem<NT, POL>& S, const XReg& X) {
    S.mask = X.mask;
    S.xok = X.xok;
    S.xg = X.xg;
    S.xsz = X.xsz;
    S.xL = X.xL;
    S.xprev = X.xprev;
    S.xright = X.xright;
    int64_t* c = S.wc[Smem<NT, POL>::NW];
    c[C_AOK] += X.aok;
    c[C_AFAIL] += X.afail;
    c[C_USEDG] += X.usedg;
    c[C_REQ] += X.req;
    c[C_NOSPLIT] += X.nosplit;
}

// Push the virtual remainder X at the head of its list and write its record
// (one thread).
template <int NT, int POL = 0>
HBA_DEV void materialize_x(Smem<NT, POL>& S, Rec* rec, XReg& X, bool cache = false) {
    const uint32_t b = X.xL, old = S.heads[b];
    const Rec r{mkx(X.xsz, ST_FREE), X.xprev, old, NIL};
    str(rec, X.xg, r);
    if (cache) {
        rec_copy_wait();  // no copy may still be landing in the slot
        S.hc[b] = r;
    }
    if (old != NIL) rec[old].w = X.xg;
    S.heads[b] = X.xg;
    cls_mark<NT, POL>(S, X.mask, b, true);
    if (X.xright < X.G) rec[X.xright].y = X.xg;
    X.xok = 0;
}

// ---------------------------------------------------------------------------
// The free phase (Algorithm 5 for all frees of the batch).
// ---------------------------------------------------------------------------

// Open-addressing table: granule -> lowest free index that names it.  A slot
// holds the key and the free index in one 64-bit word (granule << 32 | j),
// so that a probe is one load and duplicates of a key keep the lowest index
// with a 64-bit min.  Only valid frees (starts of in-use blocks) go in.
constexpr uint64_t GT_EMPTY = ~0ull;
struct GTable {
    uint64_t* slot;
    uint32_t mask;  // capacity - 1 (capacity: power of two >= 2 * keys)
};
HBA_DEV uint32_t gt_hash(uint32_t g, uint32_t mask) { return (g * 0x9E3779B1u >> 7) & mask; }
HBA_DEV void gt_insert_min(const GTable& t, uint32_t g, uint32_t j) {
    const uint64_t kv = (uint64_t)g << 32 | j;
    uint32_t s = gt_hash(g, t.mask);
    while (true) {
        const uint64_t old = at_cas_u64(&t.slot[s], GT_EMPTY, kv);
        if (old == GT_EMPTY) return;
        if ((uint32_t)(old >> 32) == g) {
            at_min_u64(&t.slot[s], kv);
            return;
        }
        s = (s + 1) & t.mask;
    }
}
// Lowest free index naming granule g, or NIL when g was not validly freed.
HBA_DEV uint32_t gt_find(const GTable& t, uint32_t g) {
    uint32_t s = gt_hash(g, t.mask);
    while (true) {
        const uint64_t v = t.slot[s];
        if (v == GT_EMPTY) return NIL;
        if ((uint32_t)(v >> 32) == g) return (uint32_t)v;
        s = (s + 1) & t.mask;
    }
}
// Capacity of the granule table for nf frees (slots of two words), where it
// starts (word offset, even: after the five staged words per free), and the
// shared-memory words of the free phase (gathered records 5 nf, table,
// roots, per-run maxima, run slots, run heads and flags 6 nf).
HBA_HD uint32_t gt_capacity(uint32_t nf) {
    uint32_t c = 2;
    while (c < 2 * nf) c <<= 1;
    return c;
}
// Free batches up to STAGE_MAX_FREES keep a region for the staged gathered
// records (five words per free, at the start); larger ones read the gathered
// records where they were gathered, and their run list takes its own array.
HBA_HD bool stage_layout(uint32_t nf) { return nf <= STAGE_MAX_FREES; }
HBA_HD uint32_t gt_offset(uint32_t nf) { return stage_layout(nf) ? (GATHER_WORDS * nf + 1u) & ~1u : 0u; }
HBA_HD uint32_t free_smem_words(uint32_t nf) {
    return gt_offset(nf) + 2 * gt_capacity(nf) + 6 * nf + (stage_layout(nf) ? 0u : nf) + 4;
}
// whether the gathered records of nf frees can be written straight into the
// free phase's shared-memory layout
HBA_HD bool stage_fits(uint32_t nf, uint32_t dyn_words) { return stage_layout(nf) && free_smem_words(nf) <= dyn_words; }
// Where the granule table of nf frees lives: in shared memory after the five
// staged words per free when the free phase fits there, else at the start of
// the global scratch.
HBA_HD uint64_t* gt_slots(uint32_t nf, uint32_t* dyn, uint32_t dyn_words, uint32_t* scr) {
    return reinterpret_cast<uint64_t*>(free_smem_words(nf) <= dyn_words ? dyn + gt_offset(nf) : scr);
}

constexpr uint32_t FL_WIN = 4;  // flag: this free is applied

template <int NT, int POL = 0>
HBA_DEV void free_phase(Smem<NT, POL>& S, const StepArgs& a) {
    const uint32_t nf = a.nf;
    Rec* rec = a.rec;
    const uint32_t hcap = gt_capacity(nf);
    // All working arrays in shared memory when they fit (the gathered records
    // are staged there first); otherwise in global memory, reading the
    // gathered records where the prep grid left them.
    const bool sm = free_smem_words(nf) <= S.dyn_words;
    // the gathered records are (or get staged) in shared memory: staging pays
    // for small free batches, large ones read them where they were gathered
    const bool copy = sm && stage_layout(nf);
    uint32_t* w = sm ? S.dyn : a.scr;
    uint32_t* const base = w;
    const uint32_t* gG;
    const uint32_t* gSZ;
    const uint32_t* gL;
    const uint32_t* gLL;
    const uint32_t* gRE;
    if (sm && copy) {
        gG = w; gSZ = w + nf; gL = w + 2 * nf; gLL = w + 3 * nf; gRE = w + 4 * nf;
    } else {
        const uint32_t gs = a.gstride;
        gG = a.gi; gSZ = a.gi + gs; gL = a.gi + 2 * gs; gLL = a.gi + 3 * gs; gRE = a.gi + 4 * gs;
    }
    if (sm) w += gt_offset(nf);
    GTable T{reinterpret_cast<uint64_t*>(w), hcap - 1};  // == gt_slots(nf, ...): cleared by arena_step
    uint32_t* root = w + 2 * hcap;      // pointer-jumping root (a free index)
    uint32_t* rmaxj = root + nf;        // largest free index of the run (at the root)
    uint32_t* rend = rmaxj + nf;        // right end of the run (at the root)
    uint32_t* runAt = rend + nf;        // run leader whose last free is j, or NIL
    uint32_t* lh = runAt + nf;          // leftmost block of the run's left part
    uint32_t* fl = lh + nf;             // bit0: erase L, bit1: erase R, FL_WIN
    uint32_t* runs = copy ? base + 3 * nf : fl + nf;  // run leaders in order (over gLL: read by then)
    uint32_t* ul = sm ? a.scr : fl + 2 * nf;                     // [2 nf] absorbed old free blocks

    // F1: stage the gathered records (shared-memory layout), and put the
    // valid frees into the granule table (lowest index wins).  The table was
    // cleared before the prep grid finished.
    HBA_FOR_THREADS(tid) {
        if (sm && copy && !a.staged) {
            const uint32_t gs = a.gstride;
            uint32_t* d = S.dyn;
            // four frees of a thread at a time: their 20 loads in flight together
            for (uint32_t j0 = tid; j0 < nf; j0 += 4 * NT) {
                uint32_t v[4][GATHER_WORDS];
                HBA_UNROLL
                for (int e = 0; e < 4; ++e) {
                    const uint32_t j = j0 + (uint32_t)e * NT;
                    HBA_UNROLL
                    for (uint32_t q = 0; q < GATHER_WORDS; ++q) v[e][q] = j < nf ? a.gi[q * gs + j] : 0u;
                }
                HBA_UNROLL
                for (int e = 0; e < 4; ++e) {
                    const uint32_t j = j0 + (uint32_t)e * NT;
                    if (j < nf) {
                        HBA_UNROLL
                        for (uint32_t q = 0; q < GATHER_WORDS; ++q) d[q * nf + j] = v[e][q];
                    }
                }
                HBA_PROF(9);
                HBA_UNROLL
                for (int e = 0; e < 4; ++e) {
                    const uint32_t j = j0 + (uint32_t)e * NT;
                    if (j < nf && v[e][0] != NIL) gt_insert_min(T, v[e][0], j);
                }
            }
        } else {
            for (uint32_t j = tid; j < nf; j += NT) {
                const uint32_t g = gG[j];
                if (g != NIL) gt_insert_min(T, g, j);
            }
        }
    }
    HBA_SYNC();
    HBA_PROF(1);
    // F2: winners and statuses; pred = the applied free to my left inside the
    // same run (directly adjacent, or across exactly one old free block); an
    // old free block absorbed by a run is unlinked by the applied free to its
    // right, or by the one to its left when it ends the run.
    HBA_FOR_THREADS(tid) {
        int64_t freed = 0;
        uint32_t won = 0;
        for (uint32_t j = tid; j < nf; j += NT) {
            const uint32_t g = gG[j];
            const bool win = g != NIL && gt_find(T, g) == j;
            if (a.fstat) a.fstat[j] = win ? 0 : 1;
            runAt[j] = NIL;
            if (!win) {
                root[j] = j;
                rmaxj[j] = 0;
                rend[j] = 0;
                fl[j] = 0;
                continue;
            }
            const uint32_t szf = gSZ[j], sz = sz_of(szf), L = gL[j];
            uint32_t pr = NIL, head = g, flags = FL_WIN;
            if (L != NIL) {
                const uint32_t wl = gt_find(T, L);
                if (wl != NIL) {
                    pr = wl;
                } else if (szf & F_LFREE) {
                    ul[at_add_u32(&S.nul, 1)] = L;
                    const uint32_t LL = gLL[j];
                    const uint32_t wll = LL != NIL ? gt_find(T, LL) : NIL;
                    if (wll != NIL) {
                        pr = wll;
                        flags |= 1;   // L is inside the run: erase its record
                    } else {
                        head = L;     // L starts the run
                    }
                }
            }
            uint32_t end = g + sz;
            if (szf & F_RFREE) {
                const uint32_t R = end;
                end = gRE[j];
                if (end >= S.G || gt_find(T, end) == NIL) {
                    ul[at_add_u32(&S.nul, 1)] = R;
                    flags |= 2;       // R ends the run: erase its record
                }
            }
            root[j] = pr == NIL ? j : pr;
            if (pr == NIL) {
                const uint32_t k = at_add_u32(&S.nlead, 1);
                if (k < LEAD_MAX) S.lead[k] = j;
            }
            rmaxj[j] = j;
            rend[j] = end;
            lh[j] = head;
            fl[j] = flags;
            freed += sz;
            ++won;
        }
        warp_sum(S, tid, C_USEDG, -freed);
        warp_sum(S, tid, C_FOK, won);
    }
    HBA_SYNC();
    HBA_PROF(2);
    // F3: every applied free finds its run's leader (leftmost applied free).
    // Runs are disjoint address ranges, so the leader of a free at granule g
    // is the leader with the largest granule <= g.
    const uint32_t nlead = S.nlead;
    if (nlead <= LEAD_MAX) {
        // few runs: rank the leaders by granule, then each free searches them
        HBA_FOR_THREADS(tid) {
            for (uint32_t t = tid; t < nlead; t += NT) {
                const uint32_t j = S.lead[t], g = gG[j];
                uint32_t rank = 0;
                for (uint32_t u = 0; u < nlead; ++u) rank += gG[S.lead[u]] < g;
                S.lkey[rank] = g;
                S.lsort[rank] = j;
            }
        }
        HBA_SYNC();
        HBA_FOR_THREADS(tid) {
            for (uint32_t j = tid; j < nf; j += NT) {
                if (!(fl[j] & FL_WIN)) continue;
                const uint32_t g = gG[j];
                uint32_t lo = 0, n = nlead;  // largest k with lkey[k] <= g
                while (n > 1) {
                    const uint32_t h = n / 2;
                    if (S.lkey[lo + h] <= g) lo += h;
                    n -= h;
                }
                root[j] = S.lsort[lo];
            }
        }
        HBA_SYNC();
    } else {
        // many runs: pointer jumping over the pred links.  Each pass
        // follows JUMP_HOPS links from every free before the barrier (four
        // frees of a thread at a time, so that their loads overlap).
        for (int it = 0;; ++it) {
            HBA_FOR_THREADS(tid) {
                bool ch = false;
                for (uint32_t j0 = tid; j0 < nf; j0 += 4 * NT) {
                    uint32_t r[4], r0[4];
                    HBA_UNROLL
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t j = j0 + (uint32_t)e * NT;
                        r[e] = r0[e] = root[j < nf ? j : j0];
                    }
                    HBA_UNROLL
                    for (int h = 0; h < JUMP_HOPS; ++h) {
                        HBA_UNROLL
                        for (int e = 0; e < 4; ++e) r[e] = root[r[e]];
                    }
                    HBA_UNROLL
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t j = j0 + (uint32_t)e * NT;
                        if (j < nf && r[e] != r0[e]) {
                            root[j] = r[e];
                            ch = true;
                        }
                    }
                }
                if (ch) S.flag[it % 3] = 1;
                if (tid == 0) S.flag[(it + 1) % 3] = 0;
            }
            HBA_SYNC();
            HBA_PROF(10);
            if (!S.flag[it % 3]) break;
        }
    }
    HBA_PROF(3);
    // F4: per-run right end and last free index; mark absorbed blocks.  A
    // warp whose frees all belong to one run reduces them first and updates
    // the run once (long runs would otherwise serialise on one address).
    HBA_FOR_THREADS(tid) {
#ifdef HBA_EMULATE
        for (uint32_t j = tid; j < nf; j += NT) {
            const uint32_t r = root[j];
            if (r != j) {
                at_max_u32(&rmaxj[r], rmaxj[j]);
                at_max_u32(&rend[r], rend[j]);
            }
        }
#else
        for (uint32_t base = 0; base < nf; base += NT) {  // same trip count in the warp
            const uint32_t j = base + (uint32_t)tid;
            uint32_t r = NIL, mj = 0, me = 0;
            if (j < nf) {
                const uint32_t rt = root[j];
                if (rt != j) {
                    r = rt;
                    mj = rmaxj[j];
                    me = rend[j];
                }
            }
            const unsigned any = __ballot_sync(0xffffffffu, r != NIL);
            if (!any) continue;
            const uint32_t rw = __shfl_sync(0xffffffffu, r, __ffs(any) - 1);
            if (__all_sync(0xffffffffu, r == NIL || r == rw)) {
                HBA_UNROLL
                for (int o = 16; o; o >>= 1) {
                    mj = max(mj, __shfl_xor_sync(0xffffffffu, mj, o));
                    me = max(me, __shfl_xor_sync(0xffffffffu, me, o));
                }
                if ((tid & 31) == 0) {
                    at_max_u32(&rmaxj[rw], mj);
                    at_max_u32(&rend[rw], me);
                }
            } else if (r != NIL) {
                at_max_u32(&rmaxj[r], mj);
                at_max_u32(&rend[r], me);
            }
        }
#endif
        for (uint32_t i = tid; i < S.nul; i += NT) {
            const uint32_t u = ul[i];
            rec[u].x = mkx(sz_of(rec[u].x), ST_DEL);
        }
    }
    HBA_SYNC();
    HBA_PROF(4);
    // F5: unlink maximal segments of absorbed blocks from their lists.
    if (S.nul) {
        HBA_FOR_THREADS(tid) {
            for (uint32_t i = tid; i < S.nul; i += NT) {
                const uint32_t u = ul[i];
                const Rec r = ldr(rec, u);
                const uint32_t pv = r.w;
                if (pv != NIL && st_of(rec[pv].x) == ST_DEL) continue;  // not a segment start
                uint32_t n = r.z;
                uint32_t guard = 0;
                while (n != NIL && st_of(rec[n].x) == ST_DEL) {
                    n = rec[n].z;
                    if (++guard > S.G) { S.err = ERR_LIST_WALK; n = NIL; break; }
                }
                if (pv == NIL) S.heads[cls_push<POL>(sz_of(r.x))] = n;
                else rec[pv].z = n;
                if (n != NIL) rec[n].w = pv;
            }
        }
        HBA_SYNC();
    }
    HBA_PROF(5);
    // F6: write the merged blocks, erase absorbed records.
    HBA_FOR_THREADS(tid) {
        uint32_t nr = 0;
        for (uint32_t j = tid; j < nf; j += NT) {
            const uint32_t f = fl[j];
            if (!(f & FL_WIN)) continue;
            const uint32_t g = gG[j];
            if (f & 1) rec[gL[j]].x = 0;
            if (f & 2) rec[g + sz_of(gSZ[j])].x = 0;
            if (root[j] == j) {
                const uint32_t H = lh[j], end = rend[j];
                rec[H].x = mkx(end - H, ST_FREE);
                if (end < S.G) rec[end].y = H;
                runAt[rmaxj[j]] = j;
                ++nr;
                if (H != g) rec[g].x = 0;
            } else {
                rec[g].x = 0;
            }
        }
        if (nr) at_add_u32(&S.nruns, nr);
    }
    HBA_SYNC();
    HBA_PROF(6);
    uint32_t nruns;
    if (nlead <= SERIAL_PUSH_MAX) {
        // F7/F8, few runs: rank the runs by their last free index, then one
        // thread pushes the merged blocks in that order
        nruns = nlead;
        HBA_FOR_THREADS(tid) {
            for (uint32_t t = tid; t < nlead; t += NT) {
                const uint32_t j = S.lsort[t], key = rmaxj[j];
                uint32_t rank = 0;
                for (uint32_t u = 0; u < nlead; ++u) rank += rmaxj[S.lsort[u]] < key;
                S.lead[rank] = j;
            }
        }
        HBA_SYNC();
        HBA_FOR_THREADS(tid) {
            if (tid == 0) {
                for (uint32_t k = 0; k < nlead; ++k) {
                    const uint32_t j = S.lead[k];
                    const uint32_t H = lh[j];
                    const uint32_t b = cls_push<POL>(rend[j] - H);
                    const uint32_t old = S.heads[b];
                    rec[H].z = old;
                    rec[H].w = NIL;
                    if (old != NIL) rec[old].w = H;
                    S.heads[b] = H;
                }
            }
        }
        HBA_SYNC();
    } else {
        // F7: run leaders in increasing order of their last free index.
        const uint32_t per = (nf + NT - 1) / NT;
        HBA_FOR_THREADS(tid) {
            const uint32_t lo = tid * per, hi = lo + per < nf ? lo + per : nf;
            uint32_t c = 0;
            for (uint32_t j = lo; j < hi; ++j) c += runAt[j] != NIL;
            S.cnt[tid] = c;
        }
        HBA_SYNC();
        scan_excl_u32<NT, POL>(S, S.cnt, &S.flag[0]);
        nruns = S.flag[0];
        HBA_FOR_THREADS(tid) {
            const uint32_t lo = tid * per, hi = lo + per < nf ? lo + per : nf;
            uint32_t k = S.cnt[tid];
            for (uint32_t j = lo; j < hi; ++j)
                if (runAt[j] != NIL) runs[k++] = runAt[j];
        }
        HBA_SYNC();
        HBA_PROF(7);
        if constexpr (POL == 0) {
        // F8a: the merged blocks are pushed in run order.  Split that order into
        // NSEG segments; inside each, link consecutive runs of the same class.
        constexpr int NSEG = Smem<NT, POL>::NSEG;
        HBA_FOR_THREADS(tid) {
            if (tid < NSEG) {
                uint32_t* F = S.segf[tid];
                uint32_t* Lt = S.segl[tid];
                for (int b = 0; b < NBINS; ++b) F[b] = Lt[b] = NIL;
                const uint32_t ps = (nruns + NSEG - 1) / NSEG;
                const uint32_t lo = tid * ps, hi = lo + ps < nruns ? lo + ps : nruns;
                for (uint32_t k = lo; k < hi; ++k) {
                    const uint32_t j = runs[k];
                    const uint32_t H = lh[j];
                    const uint32_t b = flog2(rend[j] - H);
                    if (Lt[b] == NIL) {
                        F[b] = H;
                    } else {
                        rec[H].z = Lt[b];
                        rec[Lt[b]].w = H;
                    }
                    Lt[b] = H;
                }
            }
        }
        HBA_SYNC();
        // F8b: per class, stitch the segments in order on top of the old list.
        HBA_FOR_THREADS(tid) {
            for (int b = tid; b < NBINS; b += NT) {
                uint32_t below = S.heads[b];
                bool any = false;
                for (int sgm = 0; sgm < NSEG; ++sgm) {
                    const uint32_t f = S.segf[sgm][b];
                    if (f == NIL) continue;
                    rec[f].z = below;
                    if (below != NIL) rec[below].w = f;
                    below = S.segl[sgm][b];
                    any = true;
                }
                if (any) {
                    rec[below].w = NIL;
                    S.heads[b] = below;
                }
            }
        }
        HBA_SYNC();
        } else {
            // F8 (two-level lists, too many for per-segment arrays): each run
            // finds the previous run of its list in push order (one warp, 32
            // runs at a time, the last run seen of each list in a table that
            // borrows the head-record cache, idle here); every run then links
            // below it that run, or the list's old head; the newest run of
            // each list becomes its head.
            uint32_t* last = reinterpret_cast<uint32_t*>(S.hc);  // TL_NL entries
            HBA_FOR_THREADS(tid) {
                for (uint32_t c = tid; c < TL_NL; c += NT) last[c] = NIL;
            }
            HBA_SYNC();
            HBA_FOR_THREADS(tid) {
#ifdef HBA_EMULATE
                if (tid == 0) {
                    for (uint32_t k = 0; k < nruns; ++k) {
                        const uint32_t j = runs[k];
                        const uint32_t c = cls_push<POL>(rend[j] - lh[j]);
                        root[k] = last[c];
                        last[c] = k;
                    }
                }
#else
                if ((tid >> 5) == 0) {
                    const uint32_t lane = (uint32_t)tid & 31u;
                    for (uint32_t c0 = 0; c0 < nruns; c0 += 32) {  // same trip count in the warp
                        const uint32_t k = c0 + lane;
                        const bool v = k < nruns;
                        uint32_t c = TL_NL + lane;  // idle lanes: a list of their own
                        if (v) {
                            const uint32_t j = runs[k];
                            c = cls_push<POL>(rend[j] - lh[j]);
                        }
                        const unsigned mm = __match_any_sync(0xffffffffu, c);
                        const unsigned lower = mm & ((1u << lane) - 1u);
                        if (v) root[k] = lower ? c0 + (31u - (uint32_t)__clz(lower)) : last[c];
                        __syncwarp();
                        if (v && (mm >> lane) == 1u) last[c] = k;  // the newest of its list so far
                        __syncwarp();
                    }
                }
#endif
            }
            HBA_SYNC();
            HBA_FOR_THREADS(tid) {
                for (uint32_t k = tid; k < nruns; k += NT) {
                    const uint32_t j = runs[k];
                    const uint32_t H = lh[j];
                    const uint32_t pk = root[k];
                    const uint32_t below = pk != NIL ? lh[runs[pk]] : S.heads[cls_push<POL>(rend[j] - H)];
                    rec[H].z = below;
                    if (below != NIL) rec[below].w = H;
                }
            }
            HBA_SYNC();
            HBA_FOR_THREADS(tid) {
                for (uint32_t c = tid; c < TL_NL; c += NT) {
                    const uint32_t k = last[c];
                    if (k != NIL) {
                        const uint32_t H = lh[runs[k]];
                        rec[H].w = NIL;
                        S.heads[c] = H;
                    }
                }
            }
            HBA_SYNC();
        }
    }
    if constexpr (POL == 1) {  // the second level, from the heads
        HBA_FOR_THREADS(tid) {
            for (uint32_t f = tid; f < TL_FL; f += NT) {
                uint32_t m = 0;
                for (uint32_t sb = 0; sb < TL_SL; ++sb)
                    if (S.heads[f * TL_SL + sb] != NIL) m |= 1u << sb;
                S.tsl[f] = m;
            }
        }
        HBA_SYNC();
    }
    HBA_FOR_THREADS(tid) {
        if (tid == 0) {
            uint64_t m = 0;
            if constexpr (POL == 0) {
                for (int b = 0; b < NBINS; ++b)
                    if (S.heads[b] != NIL) m |= 1ull << b;
            } else {
                for (uint32_t f = 0; f < TL_FL; ++f)
                    if (S.tsl[f]) m |= 1ull << f;
            }
            S.mask = m;
            int64_t fok = 0;
            for (int w2 = 0; w2 <= Smem<NT, POL>::NW; ++w2) fok += S.wc[w2][C_FOK];
            single_add(S, C_FFAIL, (int64_t)nf - fok);
            // every run becomes one block
            single_add(S, C_BLOCKS, (int64_t)nruns - fok - (int64_t)S.nul);
        }
    }
    HBA_SYNC();
    HBA_PROF(8);
}

// ---------------------------------------------------------------------------
// The alloc phase (Algorithm 4 for all allocations of the batch).
// ---------------------------------------------------------------------------

// Apply request i alone against the current state (one thread, X in
// registers): the general step of Algorithm 4 -- fail, carve from X, or pop
// another list.
template <int NT, int POL = 0>
HBA_DEV void seq_request(Smem<NT, POL>& S, const StepArgs& a, XReg& X, uint32_t i, uint64_t s, uint32_t sg,
                         uint32_t c) {
    Rec* rec = a.rec;
    uint32_t k;
    if constexpr (POL == 0) {
        const uint64_t M = X.mask | (X.xok ? (1ull << X.xL) : 0ull);
        const uint64_t cand = sg ? (M >> c) << c : 0ull;
        if (!cand) {
            if (!a.prefilled) a.out[i] = FAIL64;
            ++X.afail;
            return;
        }
        k = ctz64(cand);
    } else {
        k = sg ? cls_first<NT, POL>(S, X.mask, c, X.xok, X.xL) : CLS_NONE;
        if (k == CLS_NONE) {
            if (!a.prefilled) a.out[i] = FAIL64;
            ++X.afail;
            return;
        }
    }
    if (X.xok && k == X.xL) {
        // carve the front of X
        const uint32_t start = X.xg;
        str(rec, start, Rec{mkx(sg, ST_USED), X.xprev, NIL, NIL});
        a.out[i] = (uint64_t)start << X.lg;
        X.xg += sg;
        X.xsz -= sg;
        X.xprev = start;
        if (X.xsz == 0) {
            X.xok = 0;
            if (X.xright < X.G) rec[X.xright].y = start;
            ++X.nosplit;
        } else {
            X.xL = cls_push<POL>(X.xsz);
        }
    } else {
        // pop the head of list k (its record is cached); the old X becomes a
        // listed block first
        if (X.xok) materialize_x<NT, POL>(S, rec, X, true);
        const uint32_t Y = S.heads[k];
        if (Y >= X.G) {  // bitmap and heads disagree: record, fail the request
            S.err = ERR_EMPTY_HEAD;
            cls_mark<NT, POL>(S, X.mask, k, false);
            if (!a.prefilled) a.out[i] = FAIL64;
            ++X.afail;
            return;
        }
        rec_copy_wait();
        const Rec ry = S.hc[k];
        const uint32_t nxt = ry.z;
        S.heads[k] = nxt;
        if (nxt == NIL) {
            cls_mark<NT, POL>(S, X.mask, k, false);
        } else {
            rec[nxt].w = NIL;
            rec_copy_async(&S.hc[k], rec + nxt);  // the new head, for a later pop
        }
        const uint32_t ysz = sz_of(ry.x);
        str(rec, Y, Rec{mkx(sg, ST_USED), ry.y, NIL, NIL});
        a.out[i] = (uint64_t)Y << X.lg;
        if (ysz > sg) {
            X.xok = 1;
            X.xg = Y + sg;
            X.xsz = ysz - sg;
            X.xprev = Y;
            X.xright = Y + ysz;
            X.xL = cls_push<POL>(ysz - sg);
        } else {
            ++X.nosplit;
        }
    }
    ++X.aok;
    X.usedg += sg;
    X.req += (int64_t)s;
}

// Start granule of the nearest carve lane below `tid` in this round (lanes
// are carves iff S.cls == CL_CARVE; their starts are in S.cst), or X's
// prev_adj at the start of the round when there is none.  Lanes below r are
// never carves.  GPU: ballot and shuffle inside the warp, per-warp last
// carves (S.wlast) across warps.  Call convergently.
template <int NT, int POL = 0>
HBA_DEV uint32_t prev_carve_start(Smem<NT, POL>& S, int tid, uint32_t r, bool carve, uint32_t start) {
#ifdef HBA_EMULATE
    (void)carve;
    (void)start;
    for (int t = tid - 1; t >= (int)r; --t)
        if (S.cls[t] == CL_CARVE) return S.cst[t];
    return S.c0prev;
#else
    const int lane = tid & 31, wid = tid >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, carve) & ((1u << lane) - 1u);
    const int src = m ? 31 - __clz(m) : lane;
    const uint32_t v = __shfl_sync(0xffffffffu, start, src);
    if (m) return v;
    for (int w = wid - 1; w >= (int)(r >> 5); --w)
        if (S.wlast[w] != NIL) return S.wlast[w];
    return S.c0prev;
#endif
}

// Start granule of the last carve lane in [r, e), or X's prev_adj at the
// start of the round when there is none (one thread, after the verify
// barrier: per-warp carve masks in S.wcm).
template <int NT, int POL = 0>
HBA_DEV uint32_t last_carve_below(Smem<NT, POL>& S, uint32_t r, uint32_t e) {
    if (e <= r) return S.c0prev;
    const uint32_t hi = e - 1;
    int w = (int)(hi >> 5);
    const uint32_t keep = (hi & 31) == 31 ? 0xffffffffu : ((2u << (hi & 31)) - 1u);
    const uint32_t m = S.wcm[w] & keep;
    if (m) return S.cst[w * 32 + (int)flog2(m)];
    for (--w; w >= (int)(r >> 5); --w)
        if (S.wlast[w] != NIL) return S.wlast[w];
    return S.c0prev;
}

// X's fields from lane 0 to the whole warp (after lane 0 applied a request
// alone); the counters stay with lane 0, which stores them.
HBA_DEV void x_bcast(XReg& X) {
#ifndef HBA_EMULATE
    X.mask = __shfl_sync(0xffffffffu, X.mask, 0);
    X.xok = __shfl_sync(0xffffffffu, X.xok, 0);
    X.xg = __shfl_sync(0xffffffffu, X.xg, 0);
    X.xsz = __shfl_sync(0xffffffffu, X.xsz, 0);
    X.xL = __shfl_sync(0xffffffffu, X.xL, 0);
    X.xprev = __shfl_sync(0xffffffffu, X.xprev, 0);
    X.xright = __shfl_sync(0xffffffffu, X.xright, 0);
#else
    (void)X;
#endif
}

// Lane q (an event) alone, then up to `more` further lanes one by one (one
// thread), stopping before the lane that would make more than QUIET_RUN
// lanes in a row that pop no list (carves from X and failures: the lanes
// that block-wide or warp-wide rounds resolve in parallel), or more than
// QUIET_FIRST before any further pop; returns the first lane not applied.
template <int NT, int POL = 0>
HBA_DEV uint32_t seq_run(Smem<NT, POL>& S, const StepArgs& a, XReg& X, uint32_t p, uint32_t q, uint32_t stop,
                         uint32_t more) {
    seq_request<NT, POL>(S, a, X, p + q, S.s64[q], S.sgr[q], S.ccl[q]);
    ++q;
    const uint32_t end = q + more < stop ? q + more : stop;
    uint32_t quiet = 0, quiet_max = QUIET_FIRST;
    HBA_PROF(26);
    for (; q < end; ++q) {
        const uint32_t sg = S.sgr[q], c = S.ccl[q];
        bool pop = false;
        if (sg) {
            if constexpr (POL == 0) {
                const uint64_t cand = ((X.mask | (X.xok ? (1ull << X.xL) : 0ull)) >> c) << c;
                pop = cand && !(X.xok && ctz64(cand) == X.xL);
            } else {
                const uint32_t k = cls_first<NT, POL>(S, X.mask, c, X.xok, X.xL);
                pop = k != CLS_NONE && !(X.xok && k == X.xL);
            }
        }
        if (pop) {
            quiet = 0;
            quiet_max = QUIET_RUN;  // pops do come one after another here
        } else if (++quiet > quiet_max) {
            break;
        }
        seq_request<NT, POL>(S, a, X, p + q, S.s64[q], sg, c);
        HBA_PROF(27);
    }
    return q;
}

// Lanes [q, stop) of the chunk, applied by one warp in windows of 32 lanes:
// each window is classified against X, its carve sizes scanned, and the lanes
// before its first event resolved at once; lane 0 applies the event alone.
// The same rule as the block-wide rounds, with shuffles instead of barriers.
// Stops after a window without an event (events are sparse there: the
// block-wide rounds take over).  X is replicated in the warp's registers.
// Returns the first lane not applied.
#ifdef HBA_EMULATE
template <int NT, int POL = 0>
HBA_DEV uint32_t warp_stretch(Smem<NT, POL>& S, const StepArgs& a, XReg& X, uint32_t p, uint32_t q, uint32_t stop,
                              uint32_t lane) {
    (void)lane;
    Rec* rec = a.rec;
    while (q < stop) {
        const uint32_t nl = stop - q < 32u ? stop - q : 32u;
        uint8_t cl[32];
        uint64_t P[32];
        uint32_t start[32];
        uint64_t run = 0;
        for (uint32_t l = 0; l < nl; ++l) {
            const uint32_t i = q + l, sg = S.sgr[i], c = S.ccl[i];
            cl[l] = CL_FAIL;
            if (sg) {
                if constexpr (POL == 0) {
                    const uint64_t M = X.mask | (X.xok ? (1ull << X.xL) : 0ull);
                    const uint64_t cand = (M >> c) << c;
                    if (cand) cl[l] = (X.xok && ctz64(cand) == X.xL) ? CL_CARVE : CL_OTHER;
                } else {
                    const uint32_t k = cls_first<NT, POL>(S, X.mask, c, X.xok, X.xL);
                    if (k != CLS_NONE) cl[l] = (X.xok && k == X.xL) ? CL_CARVE : CL_OTHER;
                }
            }
            run += cl[l] == CL_CARVE ? sg : 0;
            P[l] = run;
        }
        uint32_t ev = nl;
        for (uint32_t l = 0; l < nl && ev == nl; ++l) {
            const uint32_t i = q + l, sg = S.sgr[i], c = S.ccl[i];
            bool e = cl[l] == CL_OTHER;
            start[l] = NIL;
            if (cl[l] == CL_CARVE) {
                const uint64_t bc = P[l] - sg;
                start[l] = X.xg + (uint32_t)bc;
                const int64_t before = (int64_t)X.xsz - (int64_t)bc;
                if constexpr (POL == 0) {
                    uint64_t M = X.mask;
                    uint32_t Lt = 64;
                    if (before > 0) {
                        Lt = flog2((uint32_t)before);
                        M |= 1ull << Lt;
                    }
                    const uint64_t cand = (M >> c) << c;
                    if (!(cand && ctz64(cand) == Lt)) e = true;
                } else if (before <= 0 || cls_first<NT, POL>(S, X.mask, c, true, cls_push<POL>((uint32_t)before)) !=
                                       cls_push<POL>((uint32_t)before))
                    e = true;
            }
            if (e) ev = l;
        }
        uint32_t prev = X.xprev;
        uint64_t gave = 0;
        for (uint32_t l = 0; l < ev; ++l) {
            const uint32_t i = q + l;
            if (cl[l] == CL_CARVE) {
                a.out[p + i] = (uint64_t)start[l] << X.lg;
                str(rec, start[l], Rec{mkx(S.sgr[i], ST_USED), prev, NIL, NIL});
                prev = start[l];
                gave = P[l];
                ++X.aok;
                X.req += (int64_t)S.s64[i];
            } else {
                if (!a.prefilled) a.out[p + i] = FAIL64;
                ++X.afail;
            }
        }
        if (gave) {
            X.xg += (uint32_t)gave;
            X.xsz -= (uint32_t)gave;
            X.xprev = prev;
            X.usedg += (int64_t)gave;
            if (X.xsz == 0) {
                X.xok = 0;
                if (X.xright < X.G) rec[X.xright].y = X.xprev;
                ++X.nosplit;
            } else {
                X.xL = cls_push<POL>(X.xsz);
            }
        }
        q += ev;
        HBA_PROF(25);
        if (ev == nl) break;
        q = seq_run<NT, POL>(S, a, X, p, q, stop, ev == 0 ? SERIAL_LANES : 0);
    }
    return q;
}
#else
template <int NT, int POL = 0>
HBA_DEV uint32_t warp_stretch(Smem<NT, POL>& S, const StepArgs& a, XReg& X, uint32_t p, uint32_t q, uint32_t stop,
                              uint32_t lane) {
    constexpr unsigned FULL = 0xffffffffu;
    Rec* rec = a.rec;
    while (q < stop) {
        const uint32_t nl = stop - q < 32u ? stop - q : 32u;
        const uint32_t i = q + lane;
        const bool in = lane < nl;
        uint32_t sg = 0, c = 0;
        uint64_t s = 0;
        uint8_t cl = CL_NONE;
        if (in) {
            sg = S.sgr[i];
            c = S.ccl[i];
            s = S.s64[i];
            cl = CL_FAIL;
            if (sg) {
                if constexpr (POL == 0) {
                    const uint64_t M = X.mask | (X.xok ? (1ull << X.xL) : 0ull);
                    const uint64_t cand = (M >> c) << c;
                    if (cand) cl = (X.xok && ctz64(cand) == X.xL) ? CL_CARVE : CL_OTHER;
                } else {
                    const uint32_t k = cls_first<NT, POL>(S, X.mask, c, X.xok, X.xL);
                    if (k != CLS_NONE) cl = (X.xok && k == X.xL) ? CL_CARVE : CL_OTHER;
                }
            }
        }
        uint64_t P = cl == CL_CARVE ? sg : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, P, o);
            if (lane >= (uint32_t)o) P += t;
        }
        bool e = cl == CL_OTHER;
        uint32_t start = NIL;
        if (cl == CL_CARVE) {
            const uint64_t bc = P - sg;
            start = X.xg + (uint32_t)bc;
            const int64_t before = (int64_t)X.xsz - (int64_t)bc;
            if constexpr (POL == 0) {
                uint64_t M = X.mask;
                uint32_t Lt = 64;
                if (before > 0) {
                    Lt = flog2((uint32_t)before);
                    M |= 1ull << Lt;
                }
                const uint64_t cand = (M >> c) << c;
                if (!(cand && ctz64(cand) == Lt)) e = true;
            } else if (before <= 0 || cls_first<NT, POL>(S, X.mask, c, true, cls_push<POL>((uint32_t)before)) !=
                                   cls_push<POL>((uint32_t)before))
                e = true;
        }
        const unsigned eb = __ballot_sync(FULL, e);
        const uint32_t ev = eb ? (uint32_t)(__ffs(eb) - 1) : nl;
        const bool act = lane < ev;
        const bool carve = act && cl == CL_CARVE;
        const bool fail = act && cl == CL_FAIL;
        const unsigned cb = __ballot_sync(FULL, carve);
        const unsigned below = cb & ((1u << lane) - 1u);
        const uint32_t pv = __shfl_sync(FULL, start, below ? 31 - __clz(below) : 0);
        if (carve) {
            a.out[p + i] = (uint64_t)start << X.lg;
            str(rec, start, Rec{mkx(sg, ST_USED), below ? pv : X.xprev, NIL, NIL});
        }
        if (fail && !a.prefilled) a.out[p + i] = FAIL64;
        const unsigned fb = __ballot_sync(FULL, fail);
        uint64_t rq = carve ? s : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) rq += __shfl_xor_sync(FULL, rq, o);
        X.aok += __popc(cb);
        X.afail += __popc(fb);
        X.req += (int64_t)rq;
        if (cb) {
            const int top = 31 - __clz(cb);
            const uint64_t gave = __shfl_sync(FULL, P, top);
            const uint32_t last = __shfl_sync(FULL, start, top);
            X.xg += (uint32_t)gave;
            X.xsz -= (uint32_t)gave;
            X.xprev = last;
            X.usedg += (int64_t)gave;
            if (X.xsz == 0) {
                X.xok = 0;
                if (lane == 0 && X.xright < X.G) rec[X.xright].y = X.xprev;
                ++X.nosplit;
            } else {
                X.xL = cls_push<POL>(X.xsz);
            }
        }
        q += ev;
        if (lane == 0) HBA_PROF(25);
        if (ev == nl) break;
        uint32_t qn = 0;
        if (lane == 0) qn = seq_run<NT, POL>(S, a, X, p, q, stop, ev == 0 ? SERIAL_LANES : 0);
        q = __shfl_sync(FULL, qn, 0);
        x_bcast(X);
        if constexpr (POL == 1) __syncwarp();  // the second-level bitmap lane 0 changed
    }
    return q;
}
#endif

// The end of a block-wide round, by warp 0 (lane 0 alone in the host
// emulation): advance X past the carves resolved in parallel, apply the event
// lane alone, go on with warp-wide rounds when events are dense, and publish
// where the next round starts.
template <int NT, int POL = 0>
HBA_DEV void round_tail(Smem<NT, POL>& S, const StepArgs& a, uint32_t p, uint32_t r, uint32_t nres, uint32_t n_here,
                        uint32_t lane) {
    Rec* rec = a.rec;
    XReg X = x_load<NT, POL>(S);
    const int64_t gave = nres > r ? S.val[nres - 1] : 0;
    if (gave > 0) {
        X.xg = S.c0g + (uint32_t)gave;
        X.xsz = S.c0sz - (uint32_t)gave;
        X.xprev = last_carve_below<NT, POL>(S, r, nres);
        X.usedg += gave;
        if (X.xsz == 0) {
            X.xok = 0;
            if (lane == 0 && X.xright < X.G) rec[X.xright].y = X.xprev;
            ++X.nosplit;
        } else {
            X.xL = cls_push<POL>(X.xsz);
        }
    }
    uint32_t next = n_here;
    if (nres < n_here) {
        // the event lane, and when (almost) nothing came before it, the next
        // few one by one
        uint32_t qn = 0;
        if (lane == 0) qn = seq_run<NT, POL>(S, a, X, p, nres, n_here, nres - r <= SERIAL_AFTER ? SERIAL_LANES : 0);
#ifdef HBA_EMULATE
        next = qn;
#else
        next = __shfl_sync(0xffffffffu, qn, 0);
        if constexpr (POL == 1) __syncwarp();  // the second-level bitmap lane 0 changed
#endif
        x_bcast(X);
        if (next < n_here && nres - r < STRETCH_BELOW) {
            const uint32_t stop = next + STRETCH_LANES < n_here ? next + STRETCH_LANES : n_here;
            next = warp_stretch<NT, POL>(S, a, X, p, next, stop, lane);
        }
    }
    if (lane == 0) {
        x_store<NT, POL>(S, X);
        S.r = next;
        S.cont = next < n_here;
        if (!S.cont) S.p = p + n_here;
    }
}

template <int NT, int POL = 0>
HBA_DEV void alloc_phase(Smem<NT, POL>& S, const StepArgs& a) {
    const uint32_t na = a.na;
    Rec* rec = a.rec;
    const uint32_t lg = S.lg;
    const uint64_t mbm = (1ull << lg) - 1ull;
    // alloc arrays live in the dynamic shared memory (the free phase is over)
    HBA_FOR_THREADS(tid) {
        if (tid == 0) {
            uint32_t* d = S.dyn;
            S.val = reinterpret_cast<int64_t*>(d);
            S.s64 = reinterpret_cast<uint64_t*>(d + 2 * NT);
            S.stg = reinterpret_cast<uint64_t*>(d + 4 * NT);
            S.cst = d + 8 * NT;
            S.sgr = d + 9 * NT;
            S.cls = reinterpret_cast<uint8_t*>(d + 10 * NT);
            S.ccl = reinterpret_cast<typename Smem<NT, POL>::ccl_t*>(d + 10 * NT + NT / 4 + 4);
            S.p = 0;
            S.xok = 0;
            // the record of every list head, for the pops of this phase
            if constexpr (POL == 0) {
                for (int b = 0; b < NBINS; ++b)
                    if (S.heads[b] != NIL) rec_copy_async(&S.hc[b], rec + S.heads[b]);
            } else {  // the non-empty lists, from the two bitmap levels
                for (uint64_t fm = S.mask; fm; fm &= fm - 1) {
                    const uint32_t f = ctz64(fm);
                    for (uint32_t sm = S.tsl[f]; sm; sm &= sm - 1) {
                        const uint32_t b = (f << TL_SLB) + ctz64(sm);
                        rec_copy_async(&S.hc[b], rec + S.heads[b]);
                    }
                }
            }
        }
    }
    HBA_SYNC();
    // the first chunk's request sizes, copied in while the loop starts
    HBA_FOR_THREADS(tid) {
        if ((uint32_t)tid < na) u64_copy_async(&S.stg[tid], a.sizes + tid);
    }
    while (true) {
        const uint32_t p = S.p;
        if (p >= na) break;
        if (!S.xok && S.mask == 0) {
            // nothing is free: every remaining request fails
            HBA_FOR_THREADS(tid) {
                if (!a.prefilled) {
#ifdef HBA_EMULATE
                    for (uint32_t i = p + tid; i < na; i += NT) a.out[i] = FAIL64;
#else
                    uint32_t lo = p;
                    if (((uintptr_t)(a.out + lo) & 15) && lo < na) {
                        if (tid == 0) a.out[lo] = FAIL64;
                        ++lo;
                    }
                    ulonglong2* o2 = reinterpret_cast<ulonglong2*>(a.out + lo);
                    const uint32_t npair = (na - lo) / 2;
                    for (uint32_t q = tid; q < npair; q += NT) o2[q] = make_ulonglong2(FAIL64, FAIL64);
                    if (((na - lo) & 1) && tid == 0) a.out[na - 1] = FAIL64;
#endif
                }
                if (tid == 0) single_add(S, C_AFAIL, (int64_t)(na - p));
            }
            HBA_SYNC();
            HBA_PROF(17);
            break;
        }
        const uint32_t n_here = na - p < (uint32_t)NT ? na - p : (uint32_t)NT;
        // Rounds over the chunk.  Each round classifies the unresolved lanes
        // [r, n_here) against the current state, assuming that every lane
        // classified as a carve from X succeeds; a lane whose true class
        // (given X's actual size in front of it) differs, or an "other", is an
        // event.  Lanes before the first event are exact and resolved in
        // parallel; the event lane is applied alone; the next round starts
        // after it.
        for (int round = 0;; ++round) {
            const uint32_t r = round == 0 ? 0u : S.r;
            uint32_t* evp = &S.evb[round & 1];
            // A: classify the lanes of the warps that hold unresolved lanes
            // (own lane only: no barrier before the scan); warps wholly
            // outside [r, n_here) sit the round out.  The first round also
            // loads the chunk (each thread its own lane, copied in ahead into
            // S.stg[chunk parity]) and starts copying the next chunk into the
            // other half.
            HBA_FOR_THREADS(tid) {
                if (round == 0) {
                    const uint32_t i = p + tid;
                    const uint32_t par = (p / NT) & 1u;
                    uint32_t sg = 0, c = 0;
                    uint64_t s = 0;
                    rec_copy_wait();
                    if (i < na) {
                        s = S.stg[par * NT + tid];
                        if (i + NT < na) u64_copy_async(&S.stg[(par ^ 1u) * NT + tid], a.sizes + i + NT);
                        if (s != 0 && s <= S.A) {
                            sg = (uint32_t)((s + mbm) >> lg);
                            c = cls_req<POL>(sg);
                        }
                    }
                    S.sgr[tid] = sg;
                    S.ccl[tid] = (typename Smem<NT, POL>::ccl_t)c;
                    S.s64[tid] = s;
                    if (tid == 0) S.evb[0] = NT;
                }
                if (warp_in_window<NT, POL>(tid >> 5, r, n_here)) {
                    uint8_t cl = CL_NONE;
                    const uint32_t sg = S.sgr[tid];
                    if ((uint32_t)tid >= r && (uint32_t)tid < n_here) {
                        if (sg == 0) {
                            cl = CL_FAIL;
                        } else {
                            const uint32_t c = S.ccl[tid];
                            if constexpr (POL == 0) {
                                const uint64_t M = S.mask | (S.xok ? (1ull << S.xL) : 0ull);
                                const uint64_t cand = (M >> c) << c;
                                if (!cand) cl = CL_FAIL;
                                else cl = (S.xok && ctz64(cand) == S.xL) ? CL_CARVE : CL_OTHER;
                            } else {
                                const uint32_t k = cls_first<NT, POL>(S, S.mask, c, S.xok, S.xL);
                                if (k == CLS_NONE) cl = CL_FAIL;
                                else cl = (S.xok && k == S.xL) ? CL_CARVE : CL_OTHER;
                            }
                        }
                    }
                    S.cls[tid] = cl;
                    S.val[tid] = cl == CL_CARVE ? (int64_t)sg : 0;
                }
                if (tid == 0) {
                    S.c0g = S.xg;
                    S.c0sz = S.xok ? S.xsz : 0;
                    S.c0prev = S.xprev;
                    S.evb[(round + 1) & 1] = NT;
                }
            }
            HBA_PROF(12);
            scan_incl_i64<NT, POL>(S, S.val, r, n_here);
            HBA_PROF(13);
            // B: verify; carve lanes record their start; per-warp carve
            // lanes and last carve
            HBA_FOR_THREADS(tid) {
                const bool wact = warp_in_window<NT, POL>(tid >> 5, r, n_here);
                if (wact) {
                    const uint8_t cl = S.cls[tid];
                    const bool carve = cl == CL_CARVE;
                    bool e = cl == CL_OTHER;
                    uint32_t start = NIL;
                    if (carve) {
                        const int64_t P = S.val[tid];
                        const uint32_t sg = S.sgr[tid];
                        start = S.c0g + (uint32_t)(P - sg);
                        const int64_t before = (int64_t)S.c0sz - (P - (int64_t)sg);
                        const uint32_t c = S.ccl[tid];
                        if constexpr (POL == 0) {
                            uint64_t M = S.mask;
                            uint32_t Lt = 64;
                            if (before > 0) {
                                Lt = flog2((uint32_t)before);
                                M |= 1ull << Lt;
                            }
                            const uint64_t cand = (M >> c) << c;
                            if (!(cand && ctz64(cand) == Lt)) e = true;
                        } else if (before <= 0 || cls_first<NT, POL>(S, S.mask, c, true, cls_push<POL>((uint32_t)before)) !=
                                               cls_push<POL>((uint32_t)before))
                            e = true;
                    }
                    S.cst[tid] = start;
#ifdef HBA_EMULATE
                    if (e && (uint32_t)tid < *evp) *evp = (uint32_t)tid;
                    if ((tid & 31) == 0) {
                        S.wcm[tid >> 5] = 0;
                        S.wlast[tid >> 5] = NIL;
                    }
                    if (carve) {
                        S.wcm[tid >> 5] |= 1u << (tid & 31);
                        S.wlast[tid >> 5] = start;
                    }
#else
                    const unsigned bal = __ballot_sync(0xffffffffu, e);
                    if ((tid & 31) == 0 && bal) atomicMin(evp, (uint32_t)(tid + __ffs(bal) - 1));
                    const unsigned cb = __ballot_sync(0xffffffffu, carve);
                    const uint32_t top = __shfl_sync(0xffffffffu, start, cb ? 31 - __clz(cb) : 0);
                    if ((tid & 31) == 0) {
                        S.wcm[tid >> 5] = cb;
                        S.wlast[tid >> 5] = cb ? top : NIL;
                    }
#endif
                } else if ((tid & 31) == 0) {
                    S.wcm[tid >> 5] = 0;
                    S.wlast[tid >> 5] = NIL;
                }
            }
            HBA_SYNC();
            HBA_PROF(14);
            const uint32_t ev = *evp;
            const uint32_t nres = ev < n_here ? ev : n_here;   // lanes [r, nres) are exact
            // C: resolve [r, nres) in parallel (failures, carves from X); then
            // warp 0 advances X past those carves, applies the event lane
            // and, when events are dense, goes on with warp-wide rounds.  The
            // events only touch records outside the carved range and results
            // of lanes >= nres, so they run beside the resolve.
            HBA_FOR_THREADS(tid) {
                if (warp_in_window<NT, POL>(tid >> 5, r, nres)) {
                    const uint8_t cl = S.cls[tid];
                    const bool act = (uint32_t)tid >= r && (uint32_t)tid < nres;
                    const bool is_fail = act && cl == CL_FAIL;
                    const bool is_carve = act && cl == CL_CARVE;
                    const uint32_t start = S.cst[tid];
                    const uint32_t prev = prev_carve_start<NT, POL>(S, tid, r, cl == CL_CARVE, start);
                    if (is_fail && !a.prefilled) a.out[p + tid] = FAIL64;
                    if (is_carve) {
                        const uint32_t sg = S.sgr[tid];
                        a.out[p + tid] = (uint64_t)start << lg;
                        str(rec, start, Rec{mkx(sg, ST_USED), prev, NIL, NIL});
                    }
                    warp_count(S, tid, C_AFAIL, is_fail);
                    warp_count(S, tid, C_AOK, is_carve);
                    warp_sum(S, tid, C_REQ, is_carve ? (int64_t)S.s64[tid] : 0);
                }
#ifdef HBA_EMULATE
                if (tid == 0) round_tail<NT, POL>(S, a, p, r, nres, n_here, 0);
#else
                if ((tid >> 5) == 0) {
                    HBA_PROF(16);
                    round_tail<NT, POL>(S, a, p, r, nres, n_here, (uint32_t)(tid & 31));
                    HBA_PROF(20);
                }
#endif
            }
            HBA_SYNC();
            HBA_PROF(15);
            if (!S.cont) break;
            if (!S.xok && S.mask == 0) {
                // nothing is free any more: the rest of the chunk fails
                HBA_FOR_THREADS(tid) {
                    const uint32_t rr = S.r;
                    const bool f = (uint32_t)tid >= rr && (uint32_t)tid < n_here;
                    if (f && !a.prefilled) a.out[p + tid] = FAIL64;
                    warp_count(S, tid, C_AFAIL, f);
                    if (tid == 0) S.p = p + n_here;
                }
                HBA_SYNC();
                break;
            }
        }
    }
    HBA_FOR_THREADS(tid) {
        if (tid == 0 && S.xok) {
            XReg X = x_load<NT, POL>(S);
            materialize_x<NT, POL>(S, rec, X);
            x_store<NT, POL>(S, X);
        }
        rec_copy_wait();  // no copy may land in shared memory after this arena
    }
    HBA_SYNC();
    HBA_PROF(18);
}

// One batch of one arena.  All threads of the CTA call this.  dyn/dyn_words:
// dynamic shared memory (at least alloc_dyn_words<NT, POL>() words).
template <int NT, int POL = 0>
HBA_DEV void arena_step(Smem<NT, POL>& S, const StepArgs& a, uint32_t* dyn, uint32_t dyn_words) {
    HBA_FOR_THREADS(tid) {
        if constexpr (POL == 0) {
            for (int b = tid; b < NBINS; b += NT) S.heads[b] = a.ar->heads[b];
        } else {
            for (uint32_t b = tid; b < TL_NL; b += NT) S.heads[b] = a.tl->heads[b];
            for (uint32_t f = tid; f < TL_FL; f += NT) S.tsl[f] = a.tl->slmask[f];
        }
        for (int q = tid; q < (Smem<NT, POL>::NW + 1) * NCNT; q += NT) (&S.wc[0][0])[q] = 0;
        if (tid == 0) {
            S.A = a.ar->arena_bytes;
            S.mask = POL ? (uint64_t)a.tl->flmask : a.ar->mask;
            S.G = a.ar->G;
            S.lg = a.ar->lg;
            S.xok = 0;
            S.xprev = NIL;
            S.nruns = 0;
            S.nul = 0;
            S.nlead = 0;
            S.flag[0] = S.flag[1] = S.flag[2] = 0;
            S.err = 0;
            S.dyn = dyn;
            S.dyn_words = dyn_words;
        }
        if (a.nf) {
            // the free phase's granule table, cleared ahead
            uint64_t* slot = gt_slots(a.nf, dyn, dyn_words, a.scr);
            const uint32_t cap = gt_capacity(a.nf);
            for (uint32_t q = tid; q < cap; q += NT) slot[q] = GT_EMPTY;
        }
    }
    HBA_SYNC();
    HBA_FOR_THREADS(tid) {
        // the first chunk's request sizes on their way to L2 (inputs: not
        // written by the preceding grid); a small arena's whole record table
        // too, so that chains of list pops do not each wait for DRAM
        const uint32_t n0 = a.na < (uint32_t)NT ? a.na : (uint32_t)NT;
        for (uint32_t q = (uint32_t)tid * 16u; q < n0; q += 16u * NT) prefetch_l2(a.sizes + q);
        if ((uint64_t)S.G * sizeof(Rec) <= PREFETCH_TABLE_MAX) {
            const uint32_t lines = (uint32_t)(((uint64_t)S.G * sizeof(Rec) + 127u) / 128u);
            for (uint32_t q = (uint32_t)tid; q < lines; q += NT)
                prefetch_l2(reinterpret_cast<const char*>(a.rec) + (size_t)q * 128u);
        }
        if (a.wait_prep == WAIT_GRID) grid_dep_wait();
        else if (a.wait_prep == WAIT_CLUSTER) cluster_wait();
    }
    StepArgs b = a;
    if (a.self_gather && a.nf) {
        // four frees a thread at a time, their record loads side by side
        const bool sm = stage_fits(a.nf, dyn_words);
        uint32_t* dst = sm ? dyn : const_cast<uint32_t*>(a.gi);
        HBA_FOR_THREADS(tid) {
            for (uint32_t j0 = tid; j0 < a.nf; j0 += 4 * NT) {
                uint64_t off[4];
                bool valid[4];
                uint32_t w[4][GATHER_WORDS];
                for (int e = 0; e < 4; ++e) {
                    const uint32_t j = j0 + (uint32_t)e * NT;
                    valid[e] = j < a.nf;
                    off[e] = valid[e] ? a.frees[j] : 0;
                }
                gather_words4(a.rec, S.A, S.G, S.lg, off, valid, w);
                for (int e = 0; e < 4; ++e) {
                    const uint32_t j = j0 + (uint32_t)e * NT;
                    if (valid[e])
                        for (uint32_t q = 0; q < GATHER_WORDS; ++q) dst[q * a.nf + j] = w[e][q];
                }
            }
        }
        HBA_SYNC();
        b.staged = sm ? 1u : 0u;
        b.gstride = a.nf;
    }
    HBA_PROF(0);
    if (b.nf) free_phase<NT, POL>(S, b);
    if (b.na) alloc_phase<NT, POL>(S, b);
    HBA_FOR_THREADS(tid) {
        if constexpr (POL == 0) {
            for (int b = tid; b < NBINS; b += NT) a.ar->heads[b] = S.heads[b];
        } else {
            for (uint32_t b = tid; b < TL_NL; b += NT) a.tl->heads[b] = S.heads[b];
            for (uint32_t f = tid; f < TL_FL; f += NT) a.tl->slmask[f] = (uint16_t)S.tsl[f];
            if (tid == 0) a.tl->flmask = (uint32_t)S.mask;
        }
        if (tid == 0) {
            int64_t c[NCNT] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int w = 0; w <= Smem<NT, POL>::NW; ++w)
                for (int k = 0; k < NCNT; ++k) c[k] += S.wc[w][k];
            Arena* ar = a.ar;
            ar->mask = S.mask;
            ar->alloc_ok += c[C_AOK];
            ar->alloc_fail += c[C_AFAIL];
            ar->free_ok += c[C_FOK];
            ar->free_fail += c[C_FFAIL];
            ar->used_g += c[C_USEDG];
            ar->used_blocks += c[C_AOK] - c[C_FOK];
            ar->blocks += c[C_AOK] - c[C_NOSPLIT] + c[C_BLOCKS];
            ar->requested += c[C_REQ];
            if (S.err && !ar->err) ar->err = S.err;
        }
    }
    HBA_SYNC();
    HBA_PROF(19);
}

// ---------------------------------------------------------------------------
// Host-side helpers shared by the library and the emulation (no device code).
// ---------------------------------------------------------------------------
inline void arena_init_host(Arena* ar, uint64_t arena_bytes, uint32_t lg, uint64_t rec_base) {
    memset(ar, 0, sizeof(*ar));
    ar->arena_bytes = arena_bytes;
    ar->rec_base = rec_base;
    ar->G = (uint32_t)(arena_bytes >> lg);
    ar->lg = lg;
    for (int b = 0; b < NBINS; ++b) ar->heads[b] = NIL;
    const uint32_t b0 = 31u - (uint32_t)__builtin_clz(ar->G);
    ar->heads[b0] = 0;
    ar->mask = 1ull << b0;
    ar->blocks = 1;
}
inline Rec initial_record(const Arena& ar) { return Rec{mkx(ar.G, ST_FREE), NIL, NIL, NIL}; }

// Canonical state (blocks in address order, lists head to tail in byte
// classes, bitmap in byte classes) from a host copy of the arena's header and
// records.  Returns the number of words; writes at most cap.
inline size_t export_canonical(const Arena& ar, const Rec* rec, uint64_t* buf, size_t cap) {
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
    for (int k = 0; k < 64; ++k) {
        const int kb = k - (int)ar.lg;
        const size_t at = n;
        put(0);
        uint64_t cnt = 0;
        if (kb >= 0 && kb < NBINS) {
            for (uint32_t h = ar.heads[kb]; h != NIL && cnt <= ar.G; ++cnt) {
                put((uint64_t)h * mb);
                h = rec[h].z;
            }
        }
        if (at < cap) buf[at] = cnt;
    }
    put(ar.mask << ar.lg);
    return n;
}

}  // namespace hba
