/* A plain C client of the library: the boundary used without Python.
 * Runs the first worked example of the test golden data (arena 4096,
 * min block 256; §5.1 Algorithms 4 and 5) through hba_alloc_batch,
 * hba_step and hba_free_batch_ex, then checks the statistics.
 * Exit status 0 when every result matches; prints what differs otherwise. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cuda_runtime.h>

#include "hba.h"

static int fails = 0;

static void expect_u64(const char* what, const uint64_t* got, const uint64_t* want, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (got[i] != want[i]) {
            printf("%s[%zu]: got %llu want %llu\n", what, i, (unsigned long long)got[i],
                   (unsigned long long)want[i]);
            ++fails;
        }
}

int main(void) {
    hba_t h = NULL;
    if (hba_create(4096, 256, HBA_POLICY_SEGFIT, &h) != HBA_OK) {
        printf("hba_create failed\n");
        return 2;
    }
    uint64_t *d_a = NULL, *d_b = NULL;
    uint8_t* d_st = NULL;
    if (cudaMalloc((void**)&d_a, 64) != cudaSuccess || cudaMalloc((void**)&d_b, 64) != cudaSuccess ||
        cudaMalloc((void**)&d_st, 8) != cudaSuccess) {
        printf("cudaMalloc failed\n");
        return 2;
    }
    uint64_t out[3];

    /* batch 1: allocations only */
    const uint64_t s1[3] = {1000, 256, 3000};
    const uint64_t w1[3] = {0, 1024, HBA_FAIL};
    cudaMemcpy(d_a, s1, sizeof s1, cudaMemcpyHostToDevice);
    if (hba_alloc_batch(h, d_a, 3, d_b, NULL) != HBA_OK) ++fails;
    cudaMemcpy(out, d_b, sizeof w1, cudaMemcpyDeviceToHost);
    expect_u64("batch 1", out, w1, 3);

    /* batch 2: one free, then one allocation, in one call */
    const uint64_t f2[1] = {0}, s2[1] = {2048}, w2[1] = {1280};
    cudaMemcpy(d_a, f2, sizeof f2, cudaMemcpyHostToDevice);
    cudaMemcpy(d_a + 4, s2, sizeof s2, cudaMemcpyHostToDevice);
    if (hba_step(h, d_a, 1, d_st, d_a + 4, 1, d_b, NULL) != HBA_OK) ++fails;
    cudaMemcpy(out, d_b, sizeof w2, cudaMemcpyDeviceToHost);
    expect_u64("batch 2", out, w2, 1);

    /* batch 3: frees through the free entry point, then an allocation */
    const uint64_t f3[2] = {1024, 1280}, s3[1] = {512}, w3[1] = {0};
    uint8_t st[2] = {9, 9};
    cudaMemcpy(d_a, f3, sizeof f3, cudaMemcpyHostToDevice);
    if (hba_free_batch_ex(h, d_a, 2, d_st, NULL) != HBA_OK) ++fails;
    cudaMemcpy(d_a + 4, s3, sizeof s3, cudaMemcpyHostToDevice);
    if (hba_alloc_batch(h, d_a + 4, 1, d_b, NULL) != HBA_OK) ++fails;
    cudaMemcpy(out, d_b, sizeof w3, cudaMemcpyDeviceToHost);
    cudaMemcpy(st, d_st, 2, cudaMemcpyDeviceToHost);
    expect_u64("batch 3", out, w3, 1);
    if (st[0] != 0 || st[1] != 0) {
        printf("batch 3 free status %u %u\n", st[0], st[1]);
        ++fails;
    }

    /* final state: [0,512) in use, [512,4096) free in byte class 11 */
    hba_stats_t sx;
    memset(&sx, 0, sizeof sx);
    if (hba_stats(h, &sx) != HBA_OK) ++fails;
    if (sx.used_bytes != 512 || sx.blocks != 2 || sx.bitmask != (1ull << 11) || sx.alloc_ok != 4 ||
        sx.alloc_fail != 1 || sx.free_ok != 3 || sx.extent_bytes != 512 || sx.largest_free != 3584) {
        printf("stats: used %llu blocks %llu bitmask %llx alloc_ok %llu alloc_fail %llu free_ok %llu "
               "extent %llu largest free %llu\n",
               (unsigned long long)sx.used_bytes, (unsigned long long)sx.blocks,
               (unsigned long long)sx.bitmask, (unsigned long long)sx.alloc_ok,
               (unsigned long long)sx.alloc_fail, (unsigned long long)sx.free_ok,
               (unsigned long long)sx.extent_bytes, (unsigned long long)sx.largest_free);
        ++fails;
    }
    hba_destroy(h);
    cudaFree(d_a);
    cudaFree(d_b);
    cudaFree(d_st);
    printf(fails ? "c client: %d mismatches\n" : "c client: ok\n", fails);
    return fails ? 1 : 0;
}
