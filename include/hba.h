/*
 * hba.h -- C ABI of the header-free batched allocator for GB300 (sm_103a).
 *
 * The allocator manages an arena of device memory that it never reads or
 * writes.  It does not even receive the arena's address: it hands out byte
 * OFFSETS into [0, arena_bytes) and takes offsets back.  All of its metadata
 * (the offset-to-block table that replaces boundary tags, the power-of-two
 * free lists and their availability bitmap) lives in separate device
 * buffers owned by the library.  This is the system model of Bell, Kumar and
 * Gill, "Host-Based Allocators for Device Memory" (arXiv 2405.07079): §1 and
 * §3 (an allocator that cannot read the memory it manages, so no boundary
 * tags), §3.3 (metadata kept out of band, keyed by block address).
 *
 * Policy.  HBA_POLICY_SEGFIT is the segregated-fit allocator of §5.1
 * (Algorithm 4 allocate, Algorithm 5 deallocate), the one the paper
 * evaluates against cudaMalloc/cudaFree in §6:
 *   - a request of `size` bytes is rounded up to s' = a multiple of
 *     min_block; its class is c = ceil(log2 s');
 *   - free blocks live in LIFO lists by floor(log2 block size); a bitmap has
 *     bit k set iff list k is non-empty;
 *   - allocation takes the head of the lowest non-empty list with index >= c
 *     (strict: list c-1 is never searched), carves s' bytes from its front and
 *     pushes the remainder, if any, at the head of its own list;
 *   - deallocation coalesces the block with a free left and/or right address
 *     neighbour and pushes the result at the head of its list.
 *
 * HBA_POLICY_TLSF is two-level segregated fit (§5.2): the same two
 * algorithms, with each power-of-two class split linearly into 16 lists (the
 * paper does not fix the count) and a second-level bitmap per class under
 * the first-level one.  A free block of z bytes is in list (floor(log2 z),
 * the four bits below the leading one); an allocation takes the head of the
 * lowest non-empty list whose lower bound is >= s' (every block there
 * fits).  TLSF handles run their batches through the same parallel batch
 * engine as segregated fit (the 512 lists with the first bitmap level in
 * the engine's bitmap word, the second level in shared memory), in the same
 * launch shapes (hba_set_shape), except that warp mode runs four arenas per
 * CTA instead of eight.  hba_serve_run rejects TLSF handles.  The canonical
 * state lists the 64 x 16 byte lists, then the first-level bitmap, then the
 * 64 second-level bitmaps.
 *
 * HBA_POLICY_FIRST_FIT, _NEXT_FIT and _BEST_FIT are the sequential fits of
 * §4 on the address-sorted free and in-use lists of §3.1 (Algorithm 1
 * allocates from the front of the chosen free block, Algorithm 2 frees and
 * coalesces).  First fit takes the lowest-address free block that fits; next
 * fit starts from the free block holding or following the end of the last
 * allocation and wraps around; best fit takes the smallest block that fits,
 * the lowest address among equal sizes.  A free at an address inside an
 * in-use block (a multiple of min_block) is a partial deallocation: the
 * block keeps its head, the tail from that address is freed.  These handles
 * run one CTA per arena, one request at a time; hba_serve_run rejects them,
 * hba_set_shape has no effect on them.  Their canonical state is the free
 * list and the in-use list as (offset, size) pairs in address order, each
 * preceded by its length, then the next-fit position, after arena and
 * min_block.
 *
 * HBA_POLICY_BITMASK is the bitmask pool of §3.2: one bit per min_block unit
 * says whether the unit is free.  An allocation of k = ceil(size / unit)
 * units (any k up to the pool; §3.2 finds 128 free bits for 1 kB at 8-byte
 * units) takes k consecutive free units by next fit (the lowest start at or
 * after the end of the last allocation, else the lowest start of all; runs
 * do not wrap).  A second out-of-band bitmap marks the first unit of
 * each in-use block; a free must name such a unit and releases the units up
 * to the next marked or free unit.  A pool holds at most 786,432 units
 * (HBA_ERR_INVALID_ARGUMENT at create); each runs on one CTA with both
 * bitmaps in shared memory.  The canonical state is the in-use blocks
 * (offset, size) in address order, preceded by their count, then the
 * next-fit position, after the pool size and the unit.
 *
 * Batch semantics.  One batch = a free call followed by an alloc call on the
 * same stream (or one hba_step call): all frees in index order, then all
 * allocations in index order, exactly as if applied one by one.  Results are
 * deterministic and bit-identical to a sequential execution of Algorithms 4
 * and 5.
 *
 * Errors.  API problems return a status (hba_status_t).  Per-request outcomes
 * are data, never errors: a failed allocation yields HBA_FAIL in its output
 * slot; a rejected free (not the start of an in-use block: unknown,
 * misaligned, interior, already free, or an earlier duplicate in the same
 * batch) yields status 1 and changes nothing.
 *
 * Streams and ownership.  Every device pointer argument is caller-owned
 * device memory that must stay valid until the work enqueued on `stream`
 * completes.  Calls are asynchronous with respect to the host unless stated
 * otherwise.  A handle's work is ordered: a call on another stream than the
 * handle's previous call waits for that call's work (an event the handle
 * records after every call; not while the stream is being captured, where
 * the caller orders).  The library allocates its metadata and scratch in
 * hba_create* and never in the batch calls.  `stream` is a cudaStream_t (NULL
 * = the legacy default stream).
 *
 * Limits.  min_block is a power of two >= 8; arena_bytes is rounded down to a
 * multiple of min_block; arena_bytes / min_block must be in [1, 2^29 - 1].
 */
#ifndef HBA_H_
#define HBA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hba_s* hba_t;
typedef void* hba_stream_t; /* a cudaStream_t */

typedef enum {
    HBA_OK = 0,
    HBA_ERR_INVALID_ARGUMENT = 1, /* bad handle, size, pointer or count */
    HBA_ERR_OUT_OF_MEMORY = 2,    /* metadata or scratch could not be allocated */
    HBA_ERR_CUDA = 3,             /* a CUDA call failed (launch, copy, sync) */
    HBA_ERR_TIMEOUT = 4,          /* a bounded device-side wait gave up */
    HBA_ERR_STATE = 5             /* the device flagged corrupted metadata */
} hba_status_t;

typedef enum {
    HBA_POLICY_SEGFIT = 0,    /* §5.1 segregated fit */
    HBA_POLICY_TLSF = 1,      /* §5.2 two-level segregated fit */
    HBA_POLICY_FIRST_FIT = 2, /* §4 first fit on address-sorted lists (§3.1) */
    HBA_POLICY_NEXT_FIT = 3,  /* §4 next fit */
    HBA_POLICY_BEST_FIT = 4,  /* §4 best fit (Algorithm 3) */
    HBA_POLICY_BITMASK = 5    /* §3.2 bitmask pool of small objects; other values are rejected */
} hba_policy_t;

#define HBA_FAIL ((uint64_t)~0ull)

/* Counters of one handle (summed over arenas for a multi-arena handle). */
typedef struct {
    uint64_t alloc_ok, alloc_fail;   /* allocations served / failed */
    uint64_t free_ok, free_fail;     /* frees applied / rejected */
    uint64_t used_bytes;             /* bytes in in-use blocks (rounded sizes) */
    uint64_t used_blocks;            /* in-use blocks */
    uint64_t blocks;                 /* all blocks, in use or free (bitmask pool: in-use
                                        blocks and maximal free runs) */
    uint64_t requested_bytes;        /* sum of the sizes of served requests */
    uint64_t free_bytes;             /* arena bytes not in use */
    uint64_t largest_free;           /* size of the largest free block (bitmask pool: the
                                        longest free run) */
    uint64_t bitmask;                /* availability bitmap (bit k: list k non-empty), arena 0;
                                        TLSF: the first level; 0 for the sequential fits and
                                        the bitmask pool */
    uint64_t arena_bytes;            /* managed bytes (sum over arenas) */
    uint64_t extent_bytes;           /* end of the highest in-use block, 0 when none (sum
                                        over arenas): the part of the arena that has to be
                                        backed by device memory, the "provisioned" memory
                                        of §6 (Fig. 4) */
    uint32_t n_arenas;
    uint32_t device_error;           /* 0, or a code the device recorded */
} hba_stats_t;

/* Create a single-arena handle on the current CUDA device (§3.3 out-of-band
 * table, §5.1 initial state: one free block [0, arena)).  Allocates the
 * offset-to-block table (16 bytes per min_block granule), scratch for
 * batches of up to 65,536 frees, and the staging and streams of the
 * host-buffer calls.  Synchronous.  *out is set only on HBA_OK. */
hba_status_t hba_create(uint64_t arena_bytes, uint64_t min_block, int policy, hba_t* out);

/* As hba_create, with scratch sized for batches of up to max_batch frees
 * (larger batches are applied in consecutive slices of max_batch, which is
 * exact because frees, like allocations, apply one by one in index order). */
hba_status_t hba_create_ex(uint64_t arena_bytes, uint64_t min_block, int policy,
                           uint32_t max_batch, hba_t* out);

/* Free all metadata of the handle.  Synchronises the device first. */
hba_status_t hba_destroy(hba_t h);

/* Allocate n blocks (Algorithm 4, one by one in index order).  d_sizes:
 * device uint64[n] of requested bytes.  d_out_offsets: device uint64[n],
 * receives the offset of each block, or HBA_FAIL.  n may be 0. */
hba_status_t hba_alloc_batch(hba_t h, const uint64_t* d_sizes, uint32_t n,
                             uint64_t* d_out_offsets, hba_stream_t stream);

/* Free n blocks (Algorithm 5, one by one in index order).  d_offsets: device
 * uint64[n].  Rejected frees are counted in the stats. */
hba_status_t hba_free_batch(hba_t h, const uint64_t* d_offsets, uint32_t n, hba_stream_t stream);

/* As hba_free_batch; d_status (device uint8[n], may be NULL) receives 0 for an
 * applied free and 1 for a rejected one. */
hba_status_t hba_free_batch_ex(hba_t h, const uint64_t* d_offsets, uint32_t n,
                               uint8_t* d_status, hba_stream_t stream);

/* One whole batch in one launch: the nf frees, then the na allocations.
 * Same results as hba_free_batch_ex followed by hba_alloc_batch. */
hba_status_t hba_step(hba_t h, const uint64_t* d_frees, uint32_t nf, uint8_t* d_status,
                      const uint64_t* d_sizes, uint32_t na, uint64_t* d_out_offsets,
                      hba_stream_t stream);

/* hba_step with HOST buffers: copies the inputs to device staging buffers,
 * runs the batch, copies the results back and waits for them.  h_status may
 * be NULL.  Staging is sized at create for max_batch requests per side;
 * larger nf or na return HBA_ERR_INVALID_ARGUMENT.  Pinned host memory gives
 * asynchronous copies; pageable memory works but is slower. */
hba_status_t hba_step_host(hba_t h, const uint64_t* h_frees, uint32_t nf, uint8_t* h_status,
                           const uint64_t* h_sizes, uint32_t na, uint64_t* h_out_offsets,
                           hba_stream_t stream);

/* hba_step_host without the host wait, for callers that keep several batches
 * in flight.  Same arguments, checks and results; returns once the work is
 * enqueued.
 *
 * Ordering.  The batch applies after every earlier call on this handle,
 * whatever its stream.  The results are in h_status / h_out_offsets once
 * `stream` reaches the point of this call: synchronise the stream, or record
 * an event on it after the call and wait for that.  The input copies do NOT
 * wait for work enqueued on `stream` before the call: h_frees and h_sizes
 * must already hold the batch when the call is made, and all four host
 * buffers must stay allocated and untouched until the results are in.  Page-
 * locked host memory is required for the copies to overlap anything.
 *
 * Pipeline.  A single-arena handle keeps two device staging slots, used in
 * turn, and three streams of its own (input copies, the engine, result
 * copies), made by hba_create with the hba_step_host staging: 50 bytes per
 * max_batch request.  Call k's input
 * copies run while call k-1's batch is on the GPU; before a slot is reused,
 * its previous results must have reached the host -- the device waits for
 * that, the host never does.
 *
 * While `stream` is being captured into a CUDA graph, the call enqueues the
 * copies and the batch on `stream` itself, in order, on the handle's
 * hba_step_host staging; the graph must then not be replayed concurrently
 * with that function. */
hba_status_t hba_step_host_async(hba_t h, const uint64_t* h_frees, uint32_t nf, uint8_t* h_status,
                                 const uint64_t* h_sizes, uint32_t na, uint64_t* h_out_offsets,
                                 hba_stream_t stream);

/* ---- batches that allocate nothing ------------------------------------- */

/* Maximum number of frees per hba_step_static call. */
#define HBA_STATIC_MAX_FREES 4096u

/* hba_step without the handle's scratch.  The paper has no counterpart: it
 * is a packaging choice of this library.
 *
 * Every handle normally carries its own device scratch for batch work,
 * allocated by hba_create* and proportional to max_batch (about 92 bytes per
 * free).  Some callers cannot afford that allocation: a process that keeps
 * many small handles under a fixed device-memory budget, or one whose device
 * memory is reserved up front by another pool, so that cudaMalloc would fail
 * or would have to be avoided.  Such callers can create their handles with
 * max_batch = 1 and run their batches here.  This call makes no allocation
 * at all: its kernels use one static device array compiled into the library
 * (room for HBA_STATIC_MAX_FREES frees, 368 KiB, held by every device
 * that loads the library until the process exits).
 *
 * Same arguments, results and stream semantics as hba_step.  nf above
 * HBA_STATIC_MAX_FREES returns HBA_ERR_INVALID_ARGUMENT and enqueues nothing.
 * The array is shared by every call on a device, whatever the handle:
 * calls whose work overlaps on the GPU (different streams without ordering
 * between them) race on it and corrupt each other's results, so order them.
 * Nothing in the array needs clearing between calls: each call writes every
 * word it reads.  The first call in each CUDA context (the device's
 * primary context, and again after cudaDeviceReset or under another
 * context) looks up the array's device address in that context and keeps it
 * for the context's later calls (HBA_ERR_CUDA if the lookup fails); make that
 * first call before any stream capture. */
hba_status_t hba_step_static(hba_t h, const uint64_t* d_frees, uint32_t nf, uint8_t* d_status,
                             const uint64_t* d_sizes, uint32_t na, uint64_t* d_out_offsets,
                             hba_stream_t stream);

/* Return the arena to its initial state (one free block) and zero the
 * counters.  Asynchronous on stream. */
hba_status_t hba_reset(hba_t h, hba_stream_t stream);

/* Read the counters and the space report (largest free block; extent, from
 * a scan of the whole record table: 16 bytes read per granule).  Waits for
 * all work on the device to finish.  Also reports HBA_ERR_STATE if the
 * device recorded a metadata error. */
hba_status_t hba_stats(hba_t h, hba_stats_t* out);

/* Canonical state of arena `arena` (0 for a single-arena handle), as 64-bit
 * words: arena_bytes, min_block, nblocks; then nblocks pairs
 * (offset, size | free << 63) in address order; then for each list k = 0..63
 * its length followed by its offsets head to tail; then the bitmap.  This is
 * the layout-independent form used to compare with a sequential reference.
 * Writes at most cap words into host_buf (may be NULL when cap is 0) and sets
 * *len to the number of words needed.  Waits for the device. */
hba_status_t hba_export_state(hba_t h, uint32_t arena, uint64_t* host_buf, size_t cap, size_t* len);

/* ---- many independent arenas in one launch ------------------------------ */

/* Create a handle over n_arenas independent arenas with the given sizes
 * (host uint64[n_arenas]), one min_block for all.  max_total_frees sizes the
 * shared scratch: the total number of frees of one hba_multi_step call. */
hba_status_t hba_multi_create(uint32_t n_arenas, const uint64_t* arena_bytes, uint64_t min_block,
                              int policy, uint32_t max_total_frees, hba_t* out);

/* One batch for every arena in one launch.  Requests are in CSR form:
 * arena a frees d_frees[d_free_rowptr[a] .. d_free_rowptr[a+1]) and allocates
 * d_sizes[d_alloc_rowptr[a] .. d_alloc_rowptr[a+1]); rowptrs are device
 * uint32[n_arenas + 1] starting at 0.  d_out is parallel to d_sizes;
 * d_free_status (may be NULL) parallel to d_frees.  The host passes the
 * totals nf_total = free_rowptr[n_arenas] and na_total = alloc_rowptr[n_arenas]
 * so that the call needs no device read-back. */
hba_status_t hba_multi_step(hba_t h, const uint32_t* d_free_rowptr, const uint64_t* d_frees,
                            uint32_t nf_total, const uint32_t* d_alloc_rowptr,
                            const uint64_t* d_sizes, uint32_t na_total, uint64_t* d_out,
                            uint8_t* d_free_status, hba_stream_t stream);

/* hba_multi_create with staging for hba_multi_step_host_async: two slots,
 * each for max_total_frees frees, max_total_allocs allocations and both
 * row-pointer arrays, allocated here (never by the calls).  max_total_allocs
 * 0 = no staging (then it is hba_multi_create). */
hba_status_t hba_multi_create_ex(uint32_t n_arenas, const uint64_t* arena_bytes, uint64_t min_block,
                                 int policy, uint32_t max_total_frees, uint32_t max_total_allocs,
                                 hba_t* out);

/* hba_multi_step from HOST buffers: the batch of every arena (same CSR
 * layout, §5.1 Algorithms 5 then 4 per arena), with the row pointers,
 * frees and sizes in host memory and the offsets (and free statuses, if
 * h_free_status is not NULL) written back to host memory.  Pipelined like
 * hba_step_host_async: the copies go through the handle's two staging slots
 * on internal streams, so call k's input copies overlap call k-1's kernels
 * and its result copies overlap call k+1's; `stream` waits for the results,
 * so synchronising it completes the call.  Returns at once; the host
 * buffers must stay untouched (inputs) and unread (outputs) until then, and
 * should be pinned for the copies to be asynchronous.  HBA_ERR_INVALID_
 * ARGUMENT if the handle has no staging (hba_multi_create) or nf_total /
 * na_total exceed max_total_frees / max_total_allocs. */
hba_status_t hba_multi_step_host_async(hba_t h, const uint32_t* h_free_rowptr, const uint64_t* h_frees,
                                       uint32_t nf_total, const uint32_t* h_alloc_rowptr,
                                       const uint64_t* h_sizes, uint32_t na_total, uint64_t* h_out,
                                       uint8_t* h_free_status, hba_stream_t stream);

/* Launch shape of the handle's batch kernel: threads per CTA (one of 64,
 * 128, 256, 512, 1024: a CTA applies one arena's batch; or 32: warp mode,
 * every warp applies its own arena's batch, 8 arenas per CTA (4 for
 * TLSF); a new
 * single-arena handle picks per batch: 128 for batches of at most 256 frees
 * and 256 allocations, else 1024); number of
 * CTAs: for a multi-arena handle, the grid (0 = enough for every arena;
 * fewer CTAs loop over the arenas); for a single-arena segregated-fit
 * handle with 256 or more threads, the size of the batch's thread-block
 * cluster (0 or 1 = no
 * cluster: a separate grid gathers the frees' records and pre-fills
 * failures, then the engine runs; 2..8 = the engine CTA plus CTAs that
 * gather the records straight into its shared memory and pre-fill failures,
 * capped at the cluster size the device holds); and dynamic
 * shared memory per CTA (per warp in warp mode) in bytes (0 = automatic: for
 * a single arena, what the batch's free phase needs; capped at the device
 * limit; a batch whose scratch does not fit uses global scratch instead).
 * Results do not depend on the shape.  Set by the autotuner or by hand. */
hba_status_t hba_set_shape(hba_t h, uint32_t threads, uint32_t ctas, uint32_t smem_bytes);

/* ---- the serving loop --------------------------------------------------- */

/* One request of an open-loop stream. */
typedef struct {
    uint64_t t_arrive_ns; /* arrival time from the start of the run; non-decreasing */
    uint64_t bytes;       /* size to allocate */
    uint64_t hold_ns;     /* how long the block is held before it is freed */
} hba_arrival_t;

/* What happened to one request. */
typedef struct {
    uint64_t offset;    /* the block, HBA_FAIL (allocation failed) or HBA_REJECTED (queue full) */
    uint64_t t_done_ns; /* device time of the result; 0 = never reached (run stopped first) */
    uint64_t t_free_ns; /* device time of its free; 0 = still held when the run ended */
} hba_served_t;

#define HBA_REJECTED ((uint64_t)~1ull)

typedef struct {
    uint32_t queue_depth;  /* admission queue capacity; 0 = 1,048,576 */
    uint32_t max_batch;    /* most frees and most allocations per tick; 0 = 4,096 */
    uint64_t bucket_ns;    /* width of a free-timing bucket; 0 = 262,144 ns */
    uint64_t time_limit_ns;/* stop after this much device time; 0 = 60 s */
    uint64_t max_ticks;    /* and after this many ticks; 0 = no limit */
} hba_serve_config_t;

typedef struct {
    uint64_t arrivals, admitted, rejected;  /* requests taken, admitted, rejected (queue full) */
    uint64_t alloc_ok, alloc_fail, frees;   /* allocator operations applied */
    uint64_t ticks, idle_ticks, max_queue;  /* loop iterations; the deepest queue */
    uint64_t elapsed_ns;                    /* device time of the run */
    uint64_t status;      /* 0 done, 1 time limit, 2 free-timing wheel full, 3 tick limit */
    uint64_t log_words;   /* words of the tick log (more than log_cap: the log is incomplete) */
} hba_serve_report_t;

/* Serve an open-loop request stream on a single-arena handle with all
 * allocator state on the device.  No counterpart in the paper (§6 runs one
 * request at a time from the host); the allocation policy is the same
 * (§5.1 Algorithms 4 and 5, through the same batch engine as hba_step).
 *
 * One persistent CTA runs ticks: it takes every request whose arrival time
 * has come (device %globaltimer) into a ring-buffer queue of queue_depth,
 * rejecting those that find it full; frees every block whose hold has ended
 * (timing by buckets of bucket_ns: a free happens at the first tick after
 * its bucket has ended); admits requests from the queue head while their
 * rounded sizes fit in the free memory; applies the tick's frees then its
 * allocations as one batch.  A request that arrives while a tick runs joins
 * the next one.
 *
 * d_arrivals: device hba_arrival_t[n].  d_served: device hba_served_t[n],
 * written by the call.  d_log (device uint32, log_cap words, may be NULL
 * with log_cap 0): per tick [nf, na, nf request ids freed, na ids admitted],
 * so that the run can be replayed exactly.  The working buffers (queue,
 * timing wheel, tick buffers: about 90 MB at the defaults) belong to the
 * handle: the first run allocates them, later runs reuse them, and a run
 * with a deeper queue or larger ticks than any before replaces them (freed
 * by hba_destroy).  Synchronous.  A run that stops at time_limit_ns
 * (report.status 1) or max_ticks (status 3) returns HBA_OK; one whose
 * timing wheel overflowed (status 2: a hold beyond 4,096 buckets, or more
 * than max_batch frees in one bucket) returns HBA_ERR_STATE, with the report
 * filled in.  The handle stays usable after any of them. */
hba_status_t hba_serve_run(hba_t h, const hba_arrival_t* d_arrivals, uint64_t n, hba_served_t* d_served,
                           uint32_t* d_log, uint64_t log_cap, const hba_serve_config_t* cfg,
                           hba_serve_report_t* report, hba_stream_t stream);

/* Version string of the library. */
const char* hba_version(void);

/* Number of kernels this handle has launched so far (batches, resets,
 * statistics, serving runs): for accounting what a timed region ran.  No
 * device work. */
hba_status_t hba_launch_count(hba_t h, uint64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* HBA_H_ */
