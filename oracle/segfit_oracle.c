/*
 * segfit_oracle.c -- sequential CPU oracle of the segregated-fit allocator
 * (Bell, Kumar, Gill, "Host-Based Allocators for Device Memory", §5.1,
 * Algorithm 4 "Allocate memory in segregated fit" and Algorithm 5
 * "Deallocate memory in segregated fit").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-sequential
 * statement of what the GPU allocator must compute.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it;
 * the library itself never links or calls it, and it shares no code,
 * header or table with the CUDA path.
 *
 * Structures are the paper's own (§3.3, §5.1):
 *   - a hash table keyed by block address whose entries hold the block size,
 *     the next/previous block of its free list, the previous adjacent block
 *     and a collision link (the six-word entry of §3.3), plus the free flag
 *     that the pseudocode of Algorithms 4/5 reads;
 *   - free_lists[64], the head address of each power-of-two size class
 *     (TLSF: 64 x 16 lists, see T1 below);
 *   - a 64-bit availability bitmap, bit k set iff list k is non-empty (§5.1).
 *
 * Readings of the pseudocode (each one is exercised by a named test):
 *   R1  class c = ceil(log2 s'), 0-based; the bin taken is the lowest set
 *       bit of the bitmap at a position >= c (Algorithm 4 with the ffs on the
 *       bitmap described after Algorithm 5).  No such bit -> the call fails.
 *   R2  strict: bin c-1 is never searched even if one of its blocks is big
 *       enough (§2.2 segregated fit: the class one magnitude larger).
 *   R3  the request is rounded up to a multiple of min_block before the class
 *       is taken and the split is made at that rounded size (§5.3 argues for
 *       a medium minimum granularity).
 *   R4  popping the head sets the new head's prev link to null and clears the
 *       bin's bit when the list becomes empty.
 *   R5  every neighbour or list-link update is skipped when its target does
 *       not exist (block at offset 0 has no left neighbour, the block ending
 *       at the arena end has no right neighbour, an empty list has no head).
 *   R6  when the left neighbour absorbs the freed block it is first unlinked
 *       from the list of its old size class; the absorbed records are erased;
 *       bins always use floor(log2 size) (Algorithm 4 split, Algorithm 5 push).
 *   R7  "right.prev = right.next" is read as "right is alone in its list":
 *       the bit is cleared when unlinking empties the list.
 *   R8  lists are LIFO stacks: push and pop at the head.
 *   R9  a failed allocation returns HBA_FAIL and changes nothing; size 0 or a
 *       rounded size above the arena fails; a free of an address that is not
 *       the start of an in-use block (unknown, interior, already free) fails
 *       and changes nothing.
 *   R10 a batch applies all frees in index order, then all allocations in
 *       index order.
 *   R11 the canonical state exported for comparison lists the blocks in
 *       address order, then each bin's list head to tail, then the bitmap.
 *
 * Two-level segregated fit (§5.2) is the same two algorithms with the
 * two-tier lookup the section describes: a first-level bitmap over the
 * power-of-two classes, each of whose bits summarises a second-level bitmap
 * that splits the class linearly into ORC_SL lists.  Readings:
 *   T1  ORC_SL = 16 lists per power of two (the paper gives no count).  The
 *       list of a block of `size` bytes is (fl, sl) with fl = floor(log2
 *       size) and sl the next four bits below the leading one: it holds the
 *       sizes [2^fl + sl 2^(fl-4), 2^fl + (sl+1) 2^(fl-4)).
 *   T2  the strict rule of R2 carries over: an allocation of s' bytes takes
 *       the lowest non-empty list whose lower bound is >= s', so that any of
 *       its blocks fits (found by rounding s' up to the next list bound, as
 *       TLSF's mapping search does, then looking at the second-level bitmap
 *       of that class and, failing that, at the first-level bitmap above it).
 *   T3  everything else (LIFO lists, splitting at s', coalescing, R3-R10) is
 *       unchanged; pushes go to the list that holds the block's size.
 *   T4  the canonical state lists the 64 x 16 lists in (fl, sl) order, then
 *       the first-level bitmap, then the 64 second-level bitmaps.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NIL UINT64_MAX   /* the "null block" that ends a list (§5.1) */
#define ORC_FAIL UINT64_MAX  /* returned by a failed allocation (R9) */
#define ORC_SEGFIT 0
#define ORC_TLSF 1
#define ORC_SL 16            /* second-level lists per power of two (T1) */
#define ORC_NLISTS (64 * ORC_SL)

typedef struct orc_entry {
    uint64_t addr;            /* key: block address (offset in the arena) */
    uint64_t size;            /* block size in bytes */
    uint64_t next_free;       /* next block in its free list, or ORC_NIL */
    uint64_t prev_free;       /* previous block in its free list, or ORC_NIL */
    uint64_t prev_adj;        /* previous adjacent block, or ORC_NIL */
    struct orc_entry* chain;  /* collision chain of the hash table */
    int free;                 /* the pseudocode's it.free */
} orc_entry;

typedef struct orc {
    uint64_t arena;           /* managed bytes, a multiple of min_block */
    uint64_t min_block;
    orc_entry** buckets;
    uint64_t nbuckets;        /* power of two */
    uint64_t count;           /* entries in the table = blocks */
    int policy;               /* ORC_SEGFIT or ORC_TLSF */
    uint64_t free_lists[ORC_NLISTS];  /* segregated fit uses the first 64 */
    uint64_t bitmask;         /* segregated fit: bit k <=> list k non-empty;
                                 TLSF: first level, bit fl <=> slmask[fl] != 0 */
    uint16_t slmask[64];      /* TLSF second level: bit sl <=> list (fl, sl) non-empty */
    /* counters reported by orc_stats */
    uint64_t alloc_ok, alloc_fail, free_ok, free_fail;
    uint64_t used_bytes, used_blocks, requested_bytes;
} orc;

/* ---- small integer helpers (library-grade primitives) ------------------ */
static unsigned floor_log2(uint64_t x) { return 63u - (unsigned)__builtin_clzll(x); }
static unsigned ceil_log2(uint64_t x) { return x <= 1 ? 0u : 64u - (unsigned)__builtin_clzll(x - 1); }

/* ---- the hash table keyed by block address (§3.3) ----------------------- */
static uint64_t bucket_of(const orc* o, uint64_t addr) {
    uint64_t h = (addr / o->min_block) * 0x9E3779B97F4A7C15ull;
    return h >> (64 - __builtin_ctzll(o->nbuckets));   /* nbuckets >= 2 */
}

static orc_entry* ht_find(const orc* o, uint64_t addr) {
    if (addr == ORC_NIL) return NULL;
    for (orc_entry* e = o->buckets[bucket_of(o, addr)]; e; e = e->chain)
        if (e->addr == addr) return e;
    return NULL;
}

static void ht_rehash(orc* o, uint64_t nb) {
    orc_entry** old = o->buckets;
    uint64_t onb = o->nbuckets;
    o->buckets = (orc_entry**)calloc(nb, sizeof(orc_entry*));
    o->nbuckets = nb;
    for (uint64_t i = 0; i < onb; i++) {
        orc_entry* e = old[i];
        while (e) {
            orc_entry* n = e->chain;
            uint64_t b = bucket_of(o, e->addr);
            e->chain = o->buckets[b];
            o->buckets[b] = e;
            e = n;
        }
    }
    free(old);
}

static orc_entry* ht_insert(orc* o, uint64_t addr) {
    if (o->count + 1 > o->nbuckets) ht_rehash(o, o->nbuckets * 2);
    orc_entry* e = (orc_entry*)calloc(1, sizeof(orc_entry));
    e->addr = addr;
    e->next_free = e->prev_free = e->prev_adj = ORC_NIL;
    uint64_t b = bucket_of(o, addr);
    e->chain = o->buckets[b];
    o->buckets[b] = e;
    o->count++;
    return e;
}

static void ht_erase(orc* o, uint64_t addr) {
    orc_entry** p = &o->buckets[bucket_of(o, addr)];
    while (*p && (*p)->addr != addr) p = &(*p)->chain;
    if (*p) {
        orc_entry* e = *p;
        *p = e->chain;
        free(e);
        o->count--;
    }
}

/* ---- free lists (LIFO, R8) --------------------------------------------- */
/* The list that holds a free block of `size` bytes: bin floor(log2 size)
 * (Algorithm 4 split, Algorithm 5 push); TLSF: fl * ORC_SL + sl (T1). */
static unsigned list_of(const orc* o, uint64_t size) {
    const unsigned fl = floor_log2(size);
    if (o->policy == ORC_SEGFIT) return fl;
    const uint64_t top = fl >= 4 ? size >> (fl - 4) : size << (4 - fl);  /* 16 + sl */
    return fl * ORC_SL + (unsigned)(top - ORC_SL);
}

static void mark(orc* o, unsigned list, int nonempty) {
    if (o->policy == ORC_SEGFIT) {
        if (nonempty) o->bitmask |= 1ull << list;
        else o->bitmask &= ~(1ull << list);
        return;
    }
    const unsigned fl = list / ORC_SL, sl = list % ORC_SL;
    if (nonempty) o->slmask[fl] |= (uint16_t)(1u << sl);
    else o->slmask[fl] &= (uint16_t)~(1u << sl);
    if (o->slmask[fl]) o->bitmask |= 1ull << fl;
    else o->bitmask &= ~(1ull << fl);
}

/* Push at the head of the block's list and set its bit (Algorithm 4 split
 * branch; Algorithm 5 final push). */
static void list_push(orc* o, orc_entry* e) {
    unsigned bin = list_of(o, e->size);
    e->next_free = o->free_lists[bin];
    e->prev_free = ORC_NIL;
    orc_entry* nx = ht_find(o, e->next_free);        /* R5: skip if empty */
    if (nx) nx->prev_free = e->addr;
    o->free_lists[bin] = e->addr;
    mark(o, bin, 1);
}

/* Remove e from the list of its size; clear the bit if the list empties
 * (Algorithm 5 remove(right) with the emptiness test of R7). */
static void list_unlink(orc* o, orc_entry* e) {
    unsigned bin = list_of(o, e->size);
    orc_entry* pv = ht_find(o, e->prev_free);
    orc_entry* nx = ht_find(o, e->next_free);
    if (pv) pv->next_free = e->next_free;
    else o->free_lists[bin] = e->next_free;
    if (nx) nx->prev_free = e->prev_free;
    if (o->free_lists[bin] == ORC_NIL) mark(o, bin, 0);
    e->next_free = e->prev_free = ORC_NIL;
}

/* The list an allocation of s bytes (rounded, R3) takes, or -1 when none
 * qualifies.  Segregated fit: the lowest set bit of the bitmap at a position
 * >= c = ceil(log2 s) (R1, R2).  TLSF (T2): round s up to the lower bound of
 * the next list (unless it is one already), take that list's (fl, sl), then
 * the lowest non-empty list at or above it: in the second-level bitmap of fl,
 * else in the first-level bitmap above fl. */
static int take_list(const orc* o, uint64_t s) {
    if (o->policy == ORC_SEGFIT) {
        unsigned c = ceil_log2(s);
        uint64_t eligible = c >= 64 ? 0 : (o->bitmask >> c) << c;
        return eligible ? __builtin_ctzll(eligible) : -1;
    }
    const unsigned f0 = floor_log2(s);
    const uint64_t r = f0 >= 4 ? s + (1ull << (f0 - 4)) - 1 : s;
    const unsigned t = list_of(o, r);
    const unsigned fl = t / ORC_SL, sl = t % ORC_SL;
    const unsigned above = o->slmask[fl] & (0xFFFFu << sl) & 0xFFFFu;
    if (above) return (int)(fl * ORC_SL + __builtin_ctz(above));
    const uint64_t fbits = fl + 1 >= 64 ? 0 : (o->bitmask >> (fl + 1)) << (fl + 1);
    if (!fbits) return -1;
    const unsigned f = (unsigned)__builtin_ctzll(fbits);
    return (int)(f * ORC_SL + __builtin_ctz(o->slmask[f]));
}

/* ---- public API -------------------------------------------------------- */
orc* orc_create_policy(uint64_t arena_bytes, uint64_t min_block, int policy) {
    if (min_block < 8 || (min_block & (min_block - 1))) return NULL;
    if (policy != ORC_SEGFIT && policy != ORC_TLSF) return NULL;
    uint64_t a = arena_bytes - arena_bytes % min_block;
    if (a == 0) return NULL;
    orc* o = (orc*)calloc(1, sizeof(orc));
    o->arena = a;
    o->min_block = min_block;
    o->policy = policy;
    o->nbuckets = 1024;
    o->buckets = (orc_entry**)calloc(o->nbuckets, sizeof(orc_entry*));
    for (int k = 0; k < ORC_NLISTS; k++) o->free_lists[k] = ORC_NIL;
    /* initial state: the whole heap is one free block (cf. §3.1, "the free
     * list always has at least one entry: the heap itself") */
    orc_entry* e = ht_insert(o, 0);
    e->size = a;
    e->free = 1;
    list_push(o, e);
    return o;
}

orc* orc_create(uint64_t arena_bytes, uint64_t min_block) {
    return orc_create_policy(arena_bytes, min_block, ORC_SEGFIT);
}

void orc_destroy(orc* o) {
    if (!o) return;
    for (uint64_t i = 0; i < o->nbuckets; i++) {
        orc_entry* e = o->buckets[i];
        while (e) { orc_entry* n = e->chain; free(e); e = n; }
    }
    free(o->buckets);
    free(o);
}

uint64_t orc_arena(const orc* o) { return o->arena; }

/* Algorithm 4 with readings R1-R5, R9. */
uint64_t orc_malloc(orc* o, uint64_t size) {
    if (size == 0 || size > o->arena) { o->alloc_fail++; return ORC_FAIL; }
    uint64_t s = (size + o->min_block - 1) / o->min_block * o->min_block;   /* R3 */
    if (s > o->arena) { o->alloc_fail++; return ORC_FAIL; }
    const int order = take_list(o, s);                                      /* R1, R2; T2 */
    if (order < 0) { o->alloc_fail++; return ORC_FAIL; }

    /* take the head of the chosen list */
    orc_entry* it = ht_find(o, o->free_lists[order]);
    list_unlink(o, it);                                                     /* R4 */
    it->free = 0;

    /* split off the surplus */
    if (s < it->size) {
        orc_entry* nb = ht_insert(o, it->addr + s);
        nb->size = it->size - s;
        nb->free = 1;
        nb->prev_adj = it->addr;
        it->size = s;
        list_push(o, nb);
        orc_entry* right = ht_find(o, nb->addr + nb->size);                 /* R5 */
        if (right) right->prev_adj = nb->addr;
    }
    o->alloc_ok++;
    o->used_bytes += it->size;
    o->used_blocks++;
    o->requested_bytes += size;
    return it->addr;
}

/* Algorithm 5 with readings R5-R7, R9.  Returns 0 on success, 1 on a
 * rejected free. */
int orc_free(orc* o, uint64_t addr) {
    orc_entry* it = ht_find(o, addr);
    if (!it || it->free) { o->free_fail++; return 1; }                      /* R9 */
    o->used_bytes -= it->size;
    o->used_blocks--;
    orc_entry* left = ht_find(o, it->prev_adj);                             /* R5 */
    orc_entry* right = it->addr + it->size < o->arena
                           ? ht_find(o, it->addr + it->size) : NULL;

    if (left && left->free) {
        list_unlink(o, left);                                               /* R6 */
        if (right && right->free) {
            /* coalesce all three, erase it and right */
            list_unlink(o, right);                                          /* R7 */
            left->size += it->size + right->size;
            orc_entry* rr = ht_find(o, right->addr + right->size);      /* R5 */
            if (rr) rr->prev_adj = left->addr;
            ht_erase(o, right->addr);
        } else {
            /* coalesce with the left block, erase it */
            left->size += it->size;
            if (right) right->prev_adj = left->addr;
        }
        ht_erase(o, it->addr);
        it = left;
    } else if (right && right->free) {
        /* coalesce with the right block */
        list_unlink(o, right);                                              /* R7 */
        it->size += right->size;
        orc_entry* rr = ht_find(o, right->addr + right->size);          /* R5 */
        if (rr) rr->prev_adj = it->addr;
        ht_erase(o, right->addr);
    }
    /* put the coalesced block at the head of its size class */
    it->free = 1;
    list_push(o, it);
    o->free_ok++;
    return 0;
}

/* One batch (R10): frees in index order, then allocations in index order.
 * free_status and out may be NULL when their counts are zero; free_status
 * may be NULL to discard the per-free status. */
void orc_batch(orc* o, const uint64_t* frees, uint32_t nf, uint8_t* free_status,
               const uint64_t* sizes, uint32_t na, uint64_t* out) {
    for (uint32_t j = 0; j < nf; j++) {
        int r = orc_free(o, frees[j]);
        if (free_status) free_status[j] = (uint8_t)r;
    }
    for (uint32_t i = 0; i < na; i++) out[i] = orc_malloc(o, sizes[i]);
}

/* Canonical state (R11, T4), as 64-bit words:
 *   arena, min_block, nblocks,
 *   nblocks pairs (offset, size | free << 63) in address order,
 *   for each list k = 0..63 (TLSF: 0..1023, k = fl * 16 + sl): count_k,
 *   then the offsets head -> tail,
 *   bitmask (TLSF: the first level), and for TLSF the 64 second-level masks.
 * Returns the number of words; writes at most cap of them. */
size_t orc_export(const orc* o, uint64_t* buf, size_t cap) {
    size_t n = 0;
#define PUT(v) do { if (n < cap) buf[n] = (v); n++; } while (0)
    PUT(o->arena);
    PUT(o->min_block);
    PUT(o->count);
    uint64_t a = 0;
    while (a < o->arena) {
        const orc_entry* e = ht_find(o, a);
        if (!e || e->size == 0) { PUT(ORC_NIL); break; }   /* broken tiling */
        PUT(e->addr);
        PUT(e->size | ((uint64_t)(e->free != 0) << 63));
        a += e->size;
    }
    const int nlists = o->policy == ORC_SEGFIT ? 64 : ORC_NLISTS;
    for (int k = 0; k < nlists; k++) {
        size_t at = n;
        PUT(0);
        uint64_t cnt = 0;
        for (uint64_t p = o->free_lists[k]; p != ORC_NIL && cnt <= o->count; cnt++) {
            const orc_entry* e = ht_find(o, p);
            if (!e) break;
            PUT(p);
            p = e->next_free;
        }
        if (at < cap) buf[at] = cnt;
    }
    PUT(o->bitmask);
    if (o->policy == ORC_TLSF)
        for (int f = 0; f < 64; f++) PUT(o->slmask[f]);
#undef PUT
    return n;
}

/* The arena's space, as §6 (Fig. 4) looks at it: out[0] = the largest free
 * block, out[1] = the extent -- the end of the highest in-use block (0 when
 * none is in use), the prefix of the arena that has to be backed by device
 * memory.  The largest free block is in the highest non-empty list, since
 * lists hold disjoint size ranges in increasing order (list k of segregated
 * fit: the sizes with floor(log2 size) = k; TLSF: T1). */
void orc_space(const orc* o, uint64_t out[2]) {
    uint64_t largest = 0, extent = 0;
    if (o->bitmask) {
        /* TLSF: the highest second-level list of the highest class */
        const unsigned f = floor_log2(o->bitmask);
        const unsigned k = o->policy == ORC_SEGFIT ? f : f * ORC_SL + floor_log2(o->slmask[f]);
        uint64_t cnt = 0;
        for (uint64_t p = o->free_lists[k]; p != ORC_NIL && cnt <= o->count; cnt++) {
            const orc_entry* e = ht_find(o, p);
            if (!e) break;
            if (e->size > largest) largest = e->size;
            p = e->next_free;
        }
    }
    for (uint64_t b = 0; b < o->nbuckets; b++)
        for (const orc_entry* e = o->buckets[b]; e; e = e->chain)
            if (!e->free && e->addr + e->size > extent) extent = e->addr + e->size;
    out[0] = largest;
    out[1] = extent;
}

/* Counters: alloc_ok, alloc_fail, free_ok, free_fail, used_bytes,
 * used_blocks, blocks, requested_bytes, bitmask. */
void orc_stats(const orc* o, uint64_t out[9]) {
    out[0] = o->alloc_ok;
    out[1] = o->alloc_fail;
    out[2] = o->free_ok;
    out[3] = o->free_fail;
    out[4] = o->used_bytes;
    out[5] = o->used_blocks;
    out[6] = o->count;
    out[7] = o->requested_bytes;
    out[8] = o->bitmask;
}
