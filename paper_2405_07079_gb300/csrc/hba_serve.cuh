// hba_serve.cuh -- the serving loop: one arena, requests arriving open-loop,
// all allocator state on the device.
//
// One persistent CTA runs ticks until the arrivals are exhausted and the
// queue is empty (or a device-time / tick limit is reached).  A tick:
//   1. takes every arrival whose time has come (device %globaltimer) into a
//      ring-buffer admission queue, rejecting those that find it full;
//   2. collects the frees that are due: successful allocations are parked in
//      a timing wheel of fixed-width buckets by the time their hold ends, and
//      every bucket that has ended is drained;
//   3. admits requests from the head of the queue while their rounded sizes
//      fit in the free memory (arena bytes in use, after this tick's frees);
//   4. applies the batch (the frees, then the admitted allocations) with the
//      same engine as every other form (arena_step: §5.1 Algorithms 5 and 4);
//   5. stamps results with the device time and logs the tick's request ids,
//      so that the run can be replayed exactly, batch by batch or one request
//      at a time.
// Requests that arrive while a tick is on the GPU join at the next tick:
// continuous batching over admission slots and free memory.  Every wait is
// bounded by the tick and time limits; the loop never spins without doing a
// tick.
#pragma once
#include "hba_engine.cuh"

namespace hba {

struct Arrival {
    uint64_t t_ns;     // arrival time, relative to the start of the run, non-decreasing
    uint64_t bytes;    // request size
    uint64_t hold_ns;  // how long the block is held before it is freed
};
struct Served {
    uint64_t offset;     // block offset, FAIL64, or REJECTED64 (queue full)
    uint64_t t_done_ns;  // when the result was produced
    uint64_t t_free_ns;  // when the block was freed (0: still held at the end)
};
constexpr uint64_t REJECTED64 = ~1ull;

// same layout as hba_serve_report_t
struct ServeCtl {
    uint64_t arrivals, admitted, rejected;
    uint64_t alloc_ok, alloc_fail, frees;
    uint64_t ticks, idle_ticks, max_queue;
    uint64_t elapsed_ns, status, log_words;
};
constexpr uint64_t SERVE_OK = 0, SERVE_TIMEOUT = 1, SERVE_WHEEL_FULL = 2, SERVE_TICK_LIMIT = 3;

struct ServeArgs {
    Arena* ar;
    Rec* rec;
    const Arrival* arr;
    uint64_t n;
    Served* served;
    uint32_t* log;
    uint64_t log_cap;
    uint32_t* queue;
    uint32_t qcap;
    uint32_t* wheel;      // W buckets x C request ids
    uint32_t* wheel_cnt;  // W counters
    uint32_t W, C;
    uint64_t bucket_ns;
    uint64_t* t_frees;    // per tick: offsets to free
    uint32_t* t_fid;      //   their request ids
    uint64_t* t_sizes;    //   sizes to allocate
    uint32_t* t_aid;      //   their request ids
    uint64_t* t_out;      //   results
    uint32_t* gi;         //   gathered records of the frees
    uint32_t* scr;        //   engine scratch
    uint32_t max_batch;
    ServeCtl* ctl;
    uint64_t time_limit_ns, max_ticks;
};

template <int NT>
struct ServeSmem {
    uint64_t now, t0, freed_bytes;
    uint64_t c_arr, c_adm, c_rej, c_ok, c_fail, c_free, c_idle, max_q;
    uint64_t cur_bucket;   // next wheel bucket (absolute number) to drain
    uint64_t log_pos;
    uint32_t a_next, q_head, q_tail, nf, na, stop, status, m;
    uint32_t nb, bfirst;   // buckets drained this tick
    uint32_t bcnt[64];     // their sizes (prefix)
    int64_t warp_tot[32];
    int64_t v[NT];
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int NT>
__device__ __forceinline__ int64_t serve_scan_incl(ServeSmem<NT>& Q, int64_t x) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) Q.warp_tot[wid] = x;
    __syncthreads();
    int64_t t = lane < NT / 32 ? Q.warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
    }
    const int64_t before = __shfl_sync(0xffffffffu, t, (wid + 31) & 31);
    if (wid > 0) x += before;
    __syncthreads();
    return x;
}

template <int NT>
__device__ void serve_loop(Smem<NT>& S, ServeSmem<NT>& Q, const ServeArgs& g, uint32_t* dyn, uint32_t dyn_words) {
    const int tid = threadIdx.x;
    const uint64_t A = g.ar->arena_bytes;
    const uint32_t lg = g.ar->lg;
    const uint64_t mbm = (1ull << lg) - 1ull;
    if (tid == 0) {
        Q.t0 = globaltimer_ns();
        Q.now = 0;
        Q.a_next = Q.q_head = Q.q_tail = 0;
        Q.c_arr = Q.c_adm = Q.c_rej = Q.c_ok = Q.c_fail = Q.c_free = Q.c_idle = Q.max_q = 0;
        Q.cur_bucket = 0;
        Q.log_pos = 0;
        Q.stop = 0;
        Q.status = SERVE_OK;
    }
    __syncthreads();
    uint64_t tick = 0;
    for (;; ++tick) {
        // 0: the clock, the limits
        if (tid == 0) {
            Q.now = globaltimer_ns() - Q.t0;
            if (Q.now > g.time_limit_ns) { Q.status = SERVE_TIMEOUT; Q.stop = 1; }
            if (g.max_ticks && tick >= g.max_ticks) { Q.status = SERVE_TICK_LIMIT; Q.stop = 1; }
            Q.nf = Q.na = 0;
            Q.freed_bytes = 0;
        }
        __syncthreads();
        if (Q.stop) break;
        HBA_PROF(40);
        const uint64_t now = Q.now;
        // 1: arrivals (sorted by time: the due ones are a prefix of each window)
        for (int pass = 0; pass < 64; ++pass) {
            const uint32_t base = Q.a_next;
            const uint64_t idx = (uint64_t)base + tid;
            const bool due = idx < g.n && g.arr[idx].t_ns <= now;
            const uint32_t m = (uint32_t)__syncthreads_count(due);
            const uint32_t qsize = Q.q_tail - Q.q_head;
            if (due) {
                if (qsize + (uint32_t)tid < g.qcap) {
                    g.queue[(Q.q_tail + (uint32_t)tid) % g.qcap] = (uint32_t)idx;
                } else {
                    g.served[idx] = Served{REJECTED64, now, 0};
                }
            }
            __syncthreads();
            if (tid == 0) {
                const uint32_t acc = qsize + m <= g.qcap ? m : g.qcap - qsize;
                Q.q_tail += acc;
                Q.c_rej += m - acc;
                Q.c_arr += m;
                Q.a_next = base + m;
                const uint64_t qs = Q.q_tail - Q.q_head;
                if (qs > Q.max_q) Q.max_q = qs;
            }
            __syncthreads();
            if (m < (uint32_t)NT) break;
        }
        HBA_PROF(41);
        // 2: due frees: every wheel bucket that has ended
        if (tid == 0) {
            uint32_t nb = 0, total = 0;
            uint64_t b = Q.cur_bucket;
            while (nb < 64 && (b + 1) * g.bucket_ns <= now) {
                const uint32_t c = g.wheel_cnt[b % g.W];
                if (total + c > g.max_batch) break;
                Q.bcnt[nb++] = total;
                total += c;
                ++b;
            }
            Q.nb = nb;
            Q.bfirst = (uint32_t)(Q.cur_bucket % g.W);
            Q.nf = total;
            Q.cur_bucket = b;
        }
        __syncthreads();
        const uint32_t nf = Q.nf, nb = Q.nb;
        int64_t fb = 0;
        for (uint32_t k = tid; k < nf; k += NT) {
            uint32_t bi = 0;
            while (bi + 1 < nb && Q.bcnt[bi + 1] <= k) ++bi;
            const uint32_t slot = (Q.bfirst + bi) % g.W;
            const uint32_t id = g.wheel[(uint64_t)slot * g.C + (k - Q.bcnt[bi])];
            g.t_fid[k] = id;
            g.t_frees[k] = g.served[id].offset;
            fb += (int64_t)((g.arr[id].bytes + mbm) & ~mbm);
        }
        fb = serve_scan_incl<NT>(Q, fb);
        if (tid == NT - 1) Q.freed_bytes = (uint64_t)fb;
        for (uint32_t bi = tid; bi < nb; bi += NT) g.wheel_cnt[(Q.bfirst + bi) % g.W] = 0;
        __syncthreads();
        HBA_PROF(42);
        // 3: admission from the queue head while the rounded sizes fit
        {
            const uint32_t qsize = Q.q_tail - Q.q_head;
            const uint32_t win = qsize < g.max_batch ? qsize : g.max_batch;
            const uint64_t used = (uint64_t)g.ar->used_g << lg;
            const uint64_t free_est = A - used + Q.freed_bytes;
            uint64_t adm_bytes = 0;   // admitted by earlier windows (same in every thread)
            uint32_t admitted = 0;
            for (uint32_t w0 = 0; w0 < win; w0 += NT) {
                const uint32_t k = w0 + tid;
                uint32_t id = 0;
                int64_t b = 0;
                if (k < win) {
                    id = g.queue[(Q.q_head + k) % g.qcap];
                    const uint64_t rb = g.arr[id].bytes;
                    b = (rb == 0 || rb > A) ? 0 : (int64_t)((rb + mbm) & ~mbm);  // invalid: admitted, fails
                }
                const int64_t pre = serve_scan_incl<NT>(Q, b);
                const bool ok = k < win && adm_bytes + (uint64_t)pre <= free_est;
                const uint32_t c = (uint32_t)__syncthreads_count(ok);  // a prefix of the window
                if (ok) {
                    g.t_aid[k] = id;
                    g.t_sizes[k] = g.arr[id].bytes;
                }
                if (c && (uint32_t)tid == c - 1) Q.freed_bytes = adm_bytes + (uint64_t)pre;  // reused as carry
                __syncthreads();
                if (c) adm_bytes = Q.freed_bytes;
                admitted += c;
                __syncthreads();
                if (c < (uint32_t)NT) break;
            }
            if (tid == 0) {
                Q.na = admitted;
                Q.q_head += admitted;
                Q.c_adm += admitted;
            }
        }
        __syncthreads();
        HBA_PROF(43);
        const uint32_t na = Q.na;
        if (nf == 0 && na == 0) {
            if (tid == 0) {
                ++Q.c_idle;
                if (Q.a_next >= g.n && Q.q_tail == Q.q_head) Q.stop = 1;
            }
            __syncthreads();
            if (Q.stop) break;
            continue;
        }
        // 4: the batch -- gather the records the frees need (four frees a
        // thread at a time, straight into the free phase's shared-memory
        // layout when it fits there), then the engine
        const bool staged = nf && stage_fits(nf, dyn_words);
        uint32_t* gdst = staged ? dyn : g.gi;
        for (uint32_t j0 = tid; j0 < nf; j0 += 4 * NT) {
            uint64_t off[4];
            bool valid[4];
            uint32_t w[4][GATHER_WORDS];
            for (int e = 0; e < 4; ++e) {
                const uint32_t j = j0 + (uint32_t)e * NT;
                valid[e] = j < nf;
                off[e] = valid[e] ? g.t_frees[j] : 0;
            }
            gather_words4(g.rec, A, g.ar->G, lg, off, valid, w);
            for (int e = 0; e < 4; ++e) {
                const uint32_t j = j0 + (uint32_t)e * NT;
                if (valid[e])
                    for (uint32_t q = 0; q < GATHER_WORDS; ++q) gdst[q * nf + j] = w[e][q];
            }
        }
        __syncthreads();
        HBA_PROF(44);
        StepArgs a{g.ar, g.rec, g.t_frees, nf, nullptr, g.t_sizes, na, g.t_out, g.scr, g.gi, nf, 0, WAIT_NONE,
                   staged ? 1u : 0u, 0};
        arena_step<NT>(S, a, dyn, dyn_words);
        if (tid == 0) Q.now = globaltimer_ns() - Q.t0;
        __syncthreads();
        HBA_PROF(45);
        const uint64_t done = Q.now;
        // 5: results, wheel, log
        int64_t ok_n = 0;
        for (uint32_t k = tid; k < na; k += NT) {
            const uint32_t id = g.t_aid[k];
            const uint64_t o = g.t_out[k];
            g.served[id] = Served{o, done, 0};
            if (o != FAIL64) {
                ++ok_n;
                const uint64_t bucket = (done + g.arr[id].hold_ns) / g.bucket_ns;
                if (bucket - Q.cur_bucket >= g.W) {
                    Q.status = SERVE_WHEEL_FULL;
                    Q.stop = 1;
                } else {
                    const uint32_t slot = (uint32_t)(bucket % g.W);
                    const uint32_t pos = atomicAdd(&g.wheel_cnt[slot], 1u);
                    if (pos < g.C) g.wheel[(uint64_t)slot * g.C + pos] = id;
                    else { Q.status = SERVE_WHEEL_FULL; Q.stop = 1; }
                }
            }
        }
        for (uint32_t k = tid; k < nf; k += NT) g.served[g.t_fid[k]].t_free_ns = done;
        ok_n = serve_scan_incl<NT>(Q, ok_n);
        if (tid == NT - 1) {
            Q.c_ok += (uint64_t)ok_n;
            Q.c_fail += na - (uint64_t)ok_n;
            Q.c_free += nf;
        }
        // log: [nf, na, free ids..., alloc ids...]
        const uint64_t lp = Q.log_pos, need = 2ull + nf + na;
        if (lp + need <= g.log_cap) {
            if (tid == 0) {
                g.log[lp] = nf;
                g.log[lp + 1] = na;
            }
            for (uint32_t k = tid; k < nf; k += NT) g.log[lp + 2 + k] = g.t_fid[k];
            for (uint32_t k = tid; k < na; k += NT) g.log[lp + 2 + nf + k] = g.t_aid[k];
        }
        __syncthreads();
        if (tid == 0) Q.log_pos = lp + need;  // past the capacity: the log is incomplete
        __syncthreads();
        HBA_PROF(46);
    }
    if (tid == 0) {
        ServeCtl* c = g.ctl;
        c->arrivals = Q.c_arr;
        c->admitted = Q.c_adm;
        c->rejected = Q.c_rej;
        c->alloc_ok = Q.c_ok;
        c->alloc_fail = Q.c_fail;
        c->frees = Q.c_free;
        c->ticks = tick;
        c->max_queue = Q.max_q;
        c->elapsed_ns = globaltimer_ns() - Q.t0;
        c->status = Q.status;
        c->log_words = Q.log_pos;
        c->idle_ticks = Q.c_idle;
    }
}

}  // namespace hba
