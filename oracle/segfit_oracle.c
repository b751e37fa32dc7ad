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
 *   - free_lists[64], the head address of each power-of-two size class;
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
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NIL UINT64_MAX   /* the "null block" that ends a list (§5.1) */
#define ORC_FAIL UINT64_MAX  /* returned by a failed allocation (R9) */

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
    uint64_t free_lists[64];
    uint64_t bitmask;
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
/* Push at the head of bin floor(log2 size) and set the bin's bit
 * (Algorithm 4 split branch; Algorithm 5 final push). */
static void list_push(orc* o, orc_entry* e) {
    unsigned bin = floor_log2(e->size);
    e->next_free = o->free_lists[bin];
    e->prev_free = ORC_NIL;
    orc_entry* nx = ht_find(o, e->next_free);        /* R5: skip if empty */
    if (nx) nx->prev_free = e->addr;
    o->free_lists[bin] = e->addr;
    o->bitmask |= 1ull << bin;
}

/* Remove e from the list of its size class; clear the bit if the list
 * empties (Algorithm 5 remove(right) with the emptiness test of R7). */
static void list_unlink(orc* o, orc_entry* e) {
    unsigned bin = floor_log2(e->size);
    orc_entry* pv = ht_find(o, e->prev_free);
    orc_entry* nx = ht_find(o, e->next_free);
    if (pv) pv->next_free = e->next_free;
    else o->free_lists[bin] = e->next_free;
    if (nx) nx->prev_free = e->prev_free;
    if (o->free_lists[bin] == ORC_NIL) o->bitmask &= ~(1ull << bin);
    e->next_free = e->prev_free = ORC_NIL;
}

/* ---- public API -------------------------------------------------------- */
orc* orc_create(uint64_t arena_bytes, uint64_t min_block) {
    if (min_block < 8 || (min_block & (min_block - 1))) return NULL;
    uint64_t a = arena_bytes - arena_bytes % min_block;
    if (a == 0) return NULL;
    orc* o = (orc*)calloc(1, sizeof(orc));
    o->arena = a;
    o->min_block = min_block;
    o->nbuckets = 1024;
    o->buckets = (orc_entry**)calloc(o->nbuckets, sizeof(orc_entry*));
    for (int k = 0; k < 64; k++) o->free_lists[k] = ORC_NIL;
    /* initial state: the whole heap is one free block (cf. §3.1, "the free
     * list always has at least one entry: the heap itself") */
    orc_entry* e = ht_insert(o, 0);
    e->size = a;
    e->free = 1;
    list_push(o, e);
    return o;
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
    unsigned c = ceil_log2(s);                                              /* R1 */
    uint64_t eligible = c >= 64 ? 0 : (o->bitmask >> c) << c;                /* R1, R2 */
    if (!eligible) { o->alloc_fail++; return ORC_FAIL; }
    unsigned order = (unsigned)__builtin_ctzll(eligible);

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

/* Canonical state (R11), as 64-bit words:
 *   arena, min_block, nblocks,
 *   nblocks pairs (offset, size | free << 63) in address order,
 *   for each bin k = 0..63: count_k, then the offsets head -> tail,
 *   bitmask.
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
    for (int k = 0; k < 64; k++) {
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
#undef PUT
    return n;
}

/* The arena's space, as §6 (Fig. 4) looks at it: out[0] = the largest free
 * block, out[1] = the extent -- the end of the highest in-use block (0 when
 * none is in use), the prefix of the arena that has to be backed by device
 * memory.  The largest free block is in the highest non-empty list, since
 * list k holds exactly the free blocks whose floor(log2 size) is k. */
void orc_space(const orc* o, uint64_t out[2]) {
    uint64_t largest = 0, extent = 0;
    if (o->bitmask) {
        const unsigned k = floor_log2(o->bitmask);
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
