/*
 * hal_oracle.c -- sequential CPU oracle of the sequential-fit allocators on
 * address-sorted lists (Bell, Kumar, Gill, "Host-Based Allocators for Device
 * Memory", §3.1 "Arrays and Hybrid Array Lists", Algorithm 1 "Memory
 * Allocation", Algorithm 2 "Memory Deallocation", §4 "Sequential Algorithms"
 * with Algorithm 3 "Best Fit Allocation" and the first-fit and next-fit
 * variants the section describes; Appendix A for the list initialisation).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never links or
 * calls it, and it shares no code, header or table with the CUDA path.
 *
 * Structures: two lists sorted by address -- the free blocks and the in-use
 * blocks -- each entry an (address, size) pair, as the HAL of §3.1 holds
 * them.  The chunked storage of a HAL (Appendix A) is a speed device that
 * does not change any result; here each list is one sorted array, searched
 * linearly, with entries shifted on insert and remove.
 *
 * Readings of the pseudocode (each one is exercised by a named test):
 *   H1  initial state: the free list holds the whole heap, the used list is
 *       empty (Appendix A initialisation; "the free list always has at
 *       least one entry: the heap itself").
 *   H2  an allocation takes the front of the chosen free block: the block
 *       [addr, addr + s') goes to the used list and the free entry moves up
 *       by s', or is removed when nothing is left (Algorithm 1).
 *   H3  sizes are rounded up to a multiple of min_block; size 0 or a
 *       rounded size above the arena fails (as R3 and R9 of segregated fit).
 *   H4  first fit: the lowest-address free block of size >= s'.
 *   H5  best fit: the smallest free block of size >= s', the lowest address
 *       among equal sizes; an exact fit ends the search.  (Algorithm 3 as
 *       printed starts its candidate at the list tail whether or not that
 *       block fits, and leaves the loop at an exact fit without taking it;
 *       both are read as the stated intent: "the smallest block that is
 *       large enough", stopping at an identical size.)
 *   H6  next fit: a roving address, 0 at start.  The search starts at the
 *       free block that contains or follows the rover (the first one whose
 *       end is above it), goes up in address order, wraps to the lowest
 *       address and stops before its starting block; the first block of
 *       size >= s' is taken, and the rover moves to the end of the
 *       allocated block ("resumes the next allocation search where the last
 *       one left off").
 *   H7  deallocation of addr finds the used block with the greatest address
 *       <= addr (Algorithm 2's search).  The free fails, changing nothing,
 *       unless addr is a multiple of min_block inside that block.  At the
 *       block's start the whole block is freed; inside it, partial
 *       deallocation frees [addr, end) and the block keeps [start, addr)
 *       ("freeing the last 2kB of a 10kB block").
 *   H8  the freed range merges with the free block that ends at its start
 *       and with the one that starts at its end (Algorithm 2's left/right
 *       tests, with adjacency meaning equality of the addresses).
 *   H9  a batch applies its frees in index order, then its allocations.
 *   H10 canonical state: the free list and the used list in address order,
 *       then the rover.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HAL_FAIL UINT64_MAX
enum { HAL_FIRST = 0, HAL_NEXT = 1, HAL_BEST = 2 };

typedef struct {
    uint64_t addr, size;
} hal_block;

typedef struct {
    hal_block* b;
    uint64_t n, cap;
} hal_list;

typedef struct hal {
    uint64_t arena, min_block;
    int fit;
    hal_list free_list, used_list;
    uint64_t rover;  /* next fit (H6) */
    uint64_t alloc_ok, alloc_fail, free_ok, free_fail, used_bytes, requested_bytes;
} hal;

/* ---- sorted lists ---------------------------------------------------------- */
static void list_insert(hal_list* l, uint64_t at, hal_block v) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 16;
        l->b = (hal_block*)realloc(l->b, l->cap * sizeof(hal_block));
    }
    memmove(l->b + at + 1, l->b + at, (l->n - at) * sizeof(hal_block));
    l->b[at] = v;
    l->n++;
}

static void list_remove(hal_list* l, uint64_t at) {
    memmove(l->b + at, l->b + at + 1, (l->n - at - 1) * sizeof(hal_block));
    l->n--;
}

/* Number of entries with address <= a (the search of Algorithm 2 returns
 * the entry before this position). */
static uint64_t count_le(const hal_list* l, uint64_t a) {
    uint64_t i = 0;
    while (i < l->n && l->b[i].addr <= a) i++;
    return i;
}

/* ---- candidate selection (§4) -------------------------------------------- */
static int64_t pick(const hal* h, uint64_t s) {
    const hal_list* f = &h->free_list;
    if (h->fit == HAL_FIRST) {                                   /* H4 */
        for (uint64_t i = 0; i < f->n; i++)
            if (f->b[i].size >= s) return (int64_t)i;
        return -1;
    }
    if (h->fit == HAL_BEST) {                                    /* H5 */
        int64_t cand = -1;
        for (uint64_t i = 0; i < f->n; i++) {
            if (f->b[i].size < s) continue;
            if (cand < 0 || f->b[i].size < f->b[cand].size) cand = (int64_t)i;
            if (f->b[i].size == s) break;
        }
        return cand;
    }
    /* next fit (H6) */
    uint64_t start = 0;
    while (start < f->n && f->b[start].addr + f->b[start].size <= h->rover) start++;
    for (uint64_t k = 0; k < f->n; k++) {
        const uint64_t i = (start + k) % f->n;
        if (f->b[i].size >= s) return (int64_t)i;
    }
    return -1;
}

/* ---- public API ------------------------------------------------------------ */
hal* hal_create(uint64_t arena_bytes, uint64_t min_block, int fit) {
    if (min_block < 8 || (min_block & (min_block - 1))) return NULL;
    if (fit != HAL_FIRST && fit != HAL_NEXT && fit != HAL_BEST) return NULL;
    uint64_t a = arena_bytes - arena_bytes % min_block;
    if (a == 0) return NULL;
    hal* h = (hal*)calloc(1, sizeof(hal));
    h->arena = a;
    h->min_block = min_block;
    h->fit = fit;
    list_insert(&h->free_list, 0, (hal_block){0, a});          /* H1 */
    return h;
}

void hal_destroy(hal* h) {
    if (!h) return;
    free(h->free_list.b);
    free(h->used_list.b);
    free(h);
}

/* Algorithm 1 on the block picked by the fit policy. */
uint64_t hal_malloc(hal* h, uint64_t size) {
    if (size == 0 || size > h->arena) { h->alloc_fail++; return HAL_FAIL; }
    const uint64_t s = (size + h->min_block - 1) / h->min_block * h->min_block;  /* H3 */
    const int64_t c = pick(h, s);
    if (c < 0) { h->alloc_fail++; return HAL_FAIL; }
    hal_block* it = &h->free_list.b[c];
    const uint64_t addr = it->addr;
    if (it->size > s) {                                         /* H2: split */
        it->addr += s;
        it->size -= s;
    } else {
        list_remove(&h->free_list, (uint64_t)c);
    }
    list_insert(&h->used_list, count_le(&h->used_list, addr), (hal_block){addr, s});
    h->rover = addr + s;
    h->alloc_ok++;
    h->used_bytes += s;
    h->requested_bytes += size;
    return addr;
}

/* Algorithm 2.  Returns 0 when applied, 1 when rejected (H7). */
int hal_free(hal* h, uint64_t addr) {
    hal_list* u = &h->used_list;
    const uint64_t p = count_le(u, addr);
    if (p == 0 || addr % h->min_block) { h->free_fail++; return 1; }
    hal_block* it = &u->b[p - 1];
    if (addr >= it->addr + it->size) { h->free_fail++; return 1; }
    uint64_t size = it->size;
    if (it->addr == addr) {
        list_remove(u, p - 1);
    } else {                                                    /* partial deallocation */
        it->size = addr - it->addr;
        size -= it->size;
    }
    h->used_bytes -= size;
    h->free_ok++;
    /* insert [addr, addr + size) into the free list, coalescing (H8) */
    hal_list* f = &h->free_list;
    const uint64_t q = count_le(f, addr);                       /* right = entry q */
    hal_block* left = q > 0 ? &f->b[q - 1] : NULL;
    hal_block* right = q < f->n ? &f->b[q] : NULL;
    const int join_left = left && left->addr + left->size == addr;
    const int join_right = right && right->addr == addr + size;
    if (join_left && join_right) {
        left->size += size + right->size;
        list_remove(f, q);
    } else if (join_left) {
        left->size += size;
    } else if (join_right) {
        right->addr = addr;
        right->size += size;
    } else {
        list_insert(f, q, (hal_block){addr, size});
    }
    return 0;
}

/* One batch (H9). */
void hal_batch(hal* h, const uint64_t* frees, uint32_t nf, uint8_t* free_status, const uint64_t* sizes,
               uint32_t na, uint64_t* out) {
    for (uint32_t j = 0; j < nf; j++) {
        const int r = hal_free(h, frees[j]);
        if (free_status) free_status[j] = (uint8_t)r;
    }
    for (uint32_t i = 0; i < na; i++) out[i] = hal_malloc(h, sizes[i]);
}

/* Canonical state (H10): arena, min_block, nfree, (addr, size) per free
 * block, nused, (addr, size) per used block, rover. */
size_t hal_export(const hal* h, uint64_t* buf, size_t cap) {
    size_t n = 0;
#define PUT(v) do { if (n < cap) buf[n] = (v); n++; } while (0)
    PUT(h->arena);
    PUT(h->min_block);
    PUT(h->free_list.n);
    for (uint64_t i = 0; i < h->free_list.n; i++) { PUT(h->free_list.b[i].addr); PUT(h->free_list.b[i].size); }
    PUT(h->used_list.n);
    for (uint64_t i = 0; i < h->used_list.n; i++) { PUT(h->used_list.b[i].addr); PUT(h->used_list.b[i].size); }
    PUT(h->rover);
#undef PUT
    return n;
}

/* alloc_ok, alloc_fail, free_ok, free_fail, used_bytes, used blocks, blocks
 * (free + used), requested_bytes, largest free block, extent (end of the
 * highest used block, 0 when none). */
void hal_stats(const hal* h, uint64_t out[10]) {
    uint64_t largest = 0;
    for (uint64_t i = 0; i < h->free_list.n; i++)
        if (h->free_list.b[i].size > largest) largest = h->free_list.b[i].size;
    const hal_list* u = &h->used_list;
    out[0] = h->alloc_ok;
    out[1] = h->alloc_fail;
    out[2] = h->free_ok;
    out[3] = h->free_fail;
    out[4] = h->used_bytes;
    out[5] = u->n;
    out[6] = u->n + h->free_list.n;
    out[7] = h->requested_bytes;
    out[8] = largest;
    out[9] = u->n ? u->b[u->n - 1].addr + u->b[u->n - 1].size : 0;
}
