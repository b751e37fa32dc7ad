/*
 * bitmask_oracle.c -- sequential CPU oracle of the bitmask pool allocator
 * (Bell, Kumar, Gill, "Host-Based Allocators for Device Memory", §3.2
 * "Bitmasks").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never links or
 * calls it, and it shares no code, header or table with the CUDA path.
 *
 * The pool is cut into units of min_block bytes.  One bit per unit says
 * whether the unit is free (§3.2: a set bit is free, allocation clears a run
 * of set bits, deallocation sets them again, so coalescing is implicit).
 *
 * Readings (each one is exercised by a named test):
 *   K1  allocation of `size` bytes needs k = ceil(size / unit) consecutive
 *       free units, for any k up to the whole pool (§3.2's own example: 1 kB
 *       at 8-byte units is a string of 128 free bits); size 0, or more units
 *       than the pool holds, fails.
 *   K2  the run is found by next fit, as §3.2 proposes: of the positions p
 *       where units [p, p + k) are all free, the lowest p at or after the
 *       rover, else (wrapping) the lowest p of all; the rover, 0 at start,
 *       moves to the end of each allocated run.  A run never wraps past the
 *       end of the pool.
 *   K3  a free names an address; the bit per unit cannot tell how many
 *       units the block had, so a second bitmap, also out of band, marks the
 *       first unit of every in-use block.  A free succeeds only at a marked
 *       unit; it frees the units from there up to the next marked unit, the
 *       next free unit or the end of the pool, whichever comes first, and
 *       clears the mark.  Anything else fails and changes nothing.
 *   K4  a batch applies its frees in index order, then its allocations.
 *   K5  canonical state: the in-use blocks (offset, size) in address order,
 *       then the rover.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BM_FAIL UINT64_MAX

typedef struct bm {
    uint64_t units, unit;     /* pool = units * unit bytes */
    uint8_t* free_bit;        /* one byte per unit here: 1 = free */
    uint8_t* start_bit;       /* 1 = first unit of an in-use block */
    uint64_t rover;           /* units */
    uint64_t alloc_ok, alloc_fail, free_ok, free_fail, used_units, requested_bytes;
} bm;

bm* bm_create(uint64_t pool_bytes, uint64_t unit) {
    if (unit < 8 || (unit & (unit - 1))) return NULL;
    const uint64_t n = pool_bytes / unit;
    if (n == 0) return NULL;
    bm* b = (bm*)calloc(1, sizeof(bm));
    b->units = n;
    b->unit = unit;
    b->free_bit = (uint8_t*)malloc(n);
    b->start_bit = (uint8_t*)calloc(n, 1);
    memset(b->free_bit, 1, n);
    return b;
}

void bm_destroy(bm* b) {
    if (!b) return;
    free(b->free_bit);
    free(b->start_bit);
    free(b);
}

/* The lowest p in [lo, hi) such that units [p, p + k) are all free and
 * p + k <= units, or UINT64_MAX: walk the units from lo, counting the free
 * units in a row; the first time the count reaches k, the string of k set
 * bits starts k - 1 units back. */
static uint64_t first_run(const bm* b, uint64_t lo, uint64_t hi, uint64_t k) {
    uint64_t run = 0;
    for (uint64_t q = lo; q < b->units; q++) {
        run = b->free_bit[q] ? run + 1 : 0;
        if (run == k) return q + 1 - k < hi ? q + 1 - k : UINT64_MAX;
    }
    return UINT64_MAX;
}

uint64_t bm_malloc(bm* b, uint64_t size) {
    const uint64_t k = size ? (size + b->unit - 1) / b->unit : 0;      /* K1 */
    if (size == 0 || size > b->units * b->unit || k > b->units) {
        b->alloc_fail++;
        return BM_FAIL;
    }
    uint64_t p = first_run(b, b->rover, b->units, k);                  /* K2 */
    if (p == UINT64_MAX) p = first_run(b, 0, b->rover, k);
    if (p == UINT64_MAX) { b->alloc_fail++; return BM_FAIL; }
    for (uint64_t q = p; q < p + k; q++) b->free_bit[q] = 0;
    b->start_bit[p] = 1;
    b->rover = p + k;
    b->alloc_ok++;
    b->used_units += k;
    b->requested_bytes += size;
    return p * b->unit;
}

int bm_free(bm* b, uint64_t addr) {
    if (addr % b->unit || addr / b->unit >= b->units || !b->start_bit[addr / b->unit]) {  /* K3 */
        b->free_fail++;
        return 1;
    }
    const uint64_t p = addr / b->unit;
    uint64_t e = p + 1;
    while (e < b->units && !b->free_bit[e] && !b->start_bit[e]) e++;
    for (uint64_t q = p; q < e; q++) b->free_bit[q] = 1;
    b->start_bit[p] = 0;
    b->free_ok++;
    b->used_units -= e - p;
    return 0;
}

void bm_batch(bm* b, const uint64_t* frees, uint32_t nf, uint8_t* free_status, const uint64_t* sizes,
              uint32_t na, uint64_t* out) {                            /* K4 */
    for (uint32_t j = 0; j < nf; j++) {
        const int r = bm_free(b, frees[j]);
        if (free_status) free_status[j] = (uint8_t)r;
    }
    for (uint32_t i = 0; i < na; i++) out[i] = bm_malloc(b, sizes[i]);
}

/* K5: pool bytes, unit, nblocks, (offset, size) per in-use block, rover (bytes). */
size_t bm_export(const bm* b, uint64_t* buf, size_t cap) {
    size_t n = 0;
#define PUT(v) do { if (n < cap) buf[n] = (v); n++; } while (0)
    PUT(b->units * b->unit);
    PUT(b->unit);
    const size_t at = n;
    PUT(0);
    uint64_t cnt = 0;
    for (uint64_t p = 0; p < b->units; p++) {
        if (!b->start_bit[p]) continue;
        uint64_t e = p + 1;
        while (e < b->units && !b->free_bit[e] && !b->start_bit[e]) e++;
        PUT(p * b->unit);
        PUT((e - p) * b->unit);
        cnt++;
    }
    if (at < cap) buf[at] = cnt;
    PUT(b->rover * b->unit);
#undef PUT
    return n;
}

/* alloc_ok, alloc_fail, free_ok, free_fail, used_bytes, used blocks, blocks
 * (in-use blocks + maximal free runs), requested_bytes, largest free run
 * (bytes), extent (end of the highest in-use unit, bytes). */
void bm_stats(const bm* b, uint64_t out[10]) {
    uint64_t used = 0, runs = 0, longest = 0, run = 0, top = 0;
    for (uint64_t p = 0; p < b->units; p++) {
        used += b->start_bit[p];
        if (b->free_bit[p]) {
            if (run == 0) runs++;
            run++;
            if (run > longest) longest = run;
        } else {
            run = 0;
            top = p + 1;
        }
    }
    out[0] = b->alloc_ok;
    out[1] = b->alloc_fail;
    out[2] = b->free_ok;
    out[3] = b->free_fail;
    out[4] = b->used_units * b->unit;
    out[5] = used;
    out[6] = used + runs;
    out[7] = b->requested_bytes;
    out[8] = longest * b->unit;
    out[9] = top * b->unit;
}
