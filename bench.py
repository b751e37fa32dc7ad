#!/usr/bin/env python3
"""Throughput of the header-free batched allocator on one GB300 (or N replicas).

Default workload (``multi``): the batched form.  4,096 independent arenas,
log-uniform 64 MiB..1 GiB (min block 256 B), each receiving U{0..2048}
requests per batch (the large trace's size mix scaled to the arena,
geometric lifetimes with mean 1,000 ops), 200 batches.  A step is one batch
of every arena: a prep grid, then one multi-arena launch.

1. The trace is recorded untimed: the seeded client drives the GPU allocator
   closed loop (it frees what the allocator gave it).
2. The launch shape is autotuned on the first batches (untimed).
3. The allocator is reset and the recorded batches are replayed: W warm-up
   steps, then K timed steps (default one pass), each bracketed by CUDA
   events on the launching stream; between steps a 256 MiB buffer is written
   to flush L2 (untimed).
4. e2e: the same replay through ``hba_multi_step_host_async`` from pinned
   host buffers, three steps in flight, the copies and the result read-back
   inside the timed region.
5. Beside it: the plain form on the same requests (one handle and launch per
   arena; results must be equal), the plain single-arena large trace, the
   oracle sharded over the host cores, and cudaMalloc / cudaMallocAsync on
   the same operations.

``--workload large|tiny|frag|usage|objects`` times the plain single-arena
form instead (one 16 GiB arena, batches of 65,536, for ``large``), with its
e2e through ``hba_step_host_async``; ``--workload serve`` the serving loop.

``--impl reference`` times the CPU oracle (the sequential statement of
Algorithms 4/5) on the same workload, one batch per step.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "alloc+free ops/s on 1 GB300 (batched/serving vs plain GPU); p50/p99 latency; bit-exact"
UNIT = "ops/s"
FAIL = np.uint64(0xFFFFFFFFFFFFFFFF)
# Algorithmic metadata bytes per request, counted with the paper's six-word
# (48-byte) address-keyed record (§3.3): a served allocation reads the list
# head and the head's record, writes it back, writes the remainder's record,
# fixes three links and the right neighbour's prev_adj (168 B with request and
# result); a failed one only reads its request and writes its result (16 B);
# an applied free reads three neighbour records and writes one plus a list
# head (216 B); a rejected free reads its request and writes a status (9 B).
BYTES_ALLOC_OK = 168
BYTES_ALLOC_FAIL = 16
BYTES_FREE_OK = 216
BYTES_FREE_REJECTED = 9
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.rows, self.proc = [], None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
        except Exception:
            sel = str(device_index)
        self.cmd = ["nvidia-smi", "-i", sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                    "-lms", "50"]

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0:  # sampler is up before timing starts
                time.sleep(0.01)
            self.rows.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        self.during = len(self.rows)
        if self.proc and not self.rows:
            # a timed region shorter than the polling period: keep the first
            # sample taken right after it
            t0 = time.time()
            while not self.rows and time.time() - t0 < 1.0:
                time.sleep(0.005)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 7
                          for i in range(4) if r[3 + i].lower() == "active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(sm)}
        if getattr(self, "during", len(sm)) == 0 and sm:
            out["note"] = "timed region shorter than the 50 ms polling period: one sample taken right after it"
        return out


def record_trace(wl, alloc, dev, space=None):
    """Drive the client closed loop against the GPU allocator (untimed).
    ``space``: a list that receives, after every batch, the memory-usage
    sample of §6 (Fig. 4): the bytes the client has live (sum of its live
    requests), the allocator's used bytes (rounded blocks), its extent (end
    of the highest in-use block: what has to be backed), and its largest
    free block and free bytes."""
    import torch

    client = wl.make()
    batches = []
    live = {}
    live_bytes = 0
    while (b := client.next_batch()) is not None:
        f, s = b
        df = torch.from_numpy(f.view(np.int64)).to(dev)
        ds = torch.from_numpy(s.view(np.int64)).to(dev)
        st = torch.empty(f.size, dtype=torch.uint8, device=dev)
        out = torch.empty(s.size, dtype=torch.int64, device=dev)
        alloc.step(df if f.size else None, ds if s.size else None, out=out, status=st)
        o = out.cpu().numpy().view(np.uint64)
        client.feed(o)
        stat = st.cpu().numpy()
        n_ok = int((o != FAIL).sum())
        n_fok = int((stat == 0).sum())
        nbytes = (BYTES_ALLOC_OK * n_ok + BYTES_ALLOC_FAIL * (s.size - n_ok)
                  + BYTES_FREE_OK * n_fok + BYTES_FREE_REJECTED * (f.size - n_fok))
        if space is not None:
            for off, fs in zip(f.tolist(), stat.tolist()):
                if fs == 0:
                    live_bytes -= live.pop(off)
            for sz, off in zip(s.tolist(), o.tolist()):
                if off != int(FAIL):
                    live[off] = sz
                    live_bytes += sz
            st_ = alloc.stats()
            space.append((live_bytes, st_["used_bytes"], st_["extent_bytes"], st_["largest_free"],
                          st_["free_bytes"]))
        batches.append({"f": df, "s": ds, "out": out, "st": st, "nf": f.size, "na": s.size,
                        "host": (f, stat, s, o),
                        "ops": f.size + s.size, "served": n_ok + n_fok, "bytes": nbytes,
                        "hf": torch.from_numpy(f.view(np.int64).copy()).pin_memory(),
                        "hs": torch.from_numpy(s.view(np.int64).copy()).pin_memory()})
    return batches


def space_report(samples, arena: int) -> dict:
    """Summary of the per-batch memory-usage samples of ``record_trace``:
    fragmentation = 1 - live / extent (the ratio §6 reads off Fig. 4: memory
    the client uses against memory that must be provisioned), the rounding
    share 1 - live / used, and largest free block / free bytes."""
    frag = [1 - lv / ex for lv, _, ex, _, _ in samples if ex]
    rnd = [1 - lv / us for lv, us, _, _, _ in samples if us]
    lff = [lf / fb for _, _, _, lf, fb in samples if fb]
    q = lambda v, p: sorted(v)[min(len(v) - 1, int(p * len(v)))] if v else None
    mean = lambda v: sum(v) / len(v) if v else None
    step = max(1, len(samples) // 16)
    return {"source": "hba_stats after every batch of the recorded trace (untimed)",
            "fragmentation": {"definition": "1 - live client bytes / extent (end of the highest in-use block)",
                              "mean": mean(frag), "p50": q(frag, 0.5), "max": max(frag) if frag else None,
                              "final": frag[-1] if frag else None},
            "rounding": {"definition": "1 - live client bytes / bytes in in-use blocks", "mean": mean(rnd)},
            "largest_free_over_free": {"mean": mean(lff), "min": min(lff) if lff else None},
            "peak_extent_bytes": max((ex for _, _, ex, _, _ in samples), default=0), "arena_bytes": arena,
            "series": {"every_batches": step, "columns": ["live_bytes", "used_bytes", "extent_bytes"],
                       "rows": [list(x[:3]) for x in samples[::step]]}}


def reduce_over_ranks(maxes, sums, world: int, device=None):
    """Whole-job figures of independent replicas: the MAX over ranks of each
    time in ``maxes`` and the SUM of each count in ``sums`` (all_reduce on the
    default process group; identity for one rank).  Returns two float lists."""
    if world <= 1:
        return [float(x) for x in maxes], [float(x) for x in sums]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


FIT_POLICIES = ("first", "next", "best")


def _make_oracle(oracle, arena, mb, policy):
    """The oracle of a policy: segregated fit / TLSF, a sequential fit, or
    the bitmask pool."""
    if policy in FIT_POLICIES:
        return oracle.HalOracle(arena, mb, policy)
    if policy == "bitmask":
        return oracle.BitmaskOracle(arena, mb)
    return oracle.Oracle(arena, mb, policy)


def _oracle_arenas(work):
    """Pool worker: the oracle over whole per-arena request sequences.
    work = list of (arena_bytes, min_block, policy, [(frees, sizes), ...]); returns
    (ops, oracle seconds, results per arena)."""
    sys.path.insert(0, ROOT)
    import oracle

    ops, secs, res = 0, 0.0, []
    for arena, mb, policy, seq in work:
        o = _make_oracle(oracle, arena, mb, policy)
        outs = []
        for f, s in seq:
            t0 = time.perf_counter()
            out, st = o.batch(f, s)
            secs += time.perf_counter() - t0
            ops += f.size + s.size
            outs.append((out, st))
        res.append(outs)
    return ops, secs, res


def oracle_pool_baseline(arenas, mb, seqs, cores=None, policy="segfit") -> tuple:
    """The oracle on independent arenas, sharded over the host's cores
    (spawned processes).  Returns (ops/s over the pool's wall time, cores,
    per-arena results)."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    cores = cores or max(1, min(len(os.sched_getaffinity(0)), len(arenas)))
    shards = [[] for _ in range(cores)]
    for i, (a, seq) in enumerate(zip(arenas, seqs)):
        shards[i % cores].append((int(a), mb, policy, seq))
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_arenas, [[] for _ in range(cores)])  # workers up before the clock starts
        t0 = time.perf_counter()
        parts = pool.map(_oracle_arenas, shards)
        wall = time.perf_counter() - t0
    ops = sum(p[0] for p in parts)
    res = [None] * len(arenas)
    for c, part in enumerate(parts):
        for k, r in enumerate(part[2]):
            res[c + k * cores] = r
    return ops / wall, cores, res


def cuda_replay_ops_multi(batches, arenas):
    """Operation list for the CUDA allocators from a batched trace: per batch,
    for each of the given arenas, its applied frees then its served
    allocations (offsets are per arena)."""
    live, ops, nslot = {}, [], 0
    for b in batches:
        fr, ar = b["hfrow"], b["harow"]
        for i in arenas:
            for j in range(int(fr[i]), int(fr[i + 1])):
                if b["ref_st"][j] == 0:
                    ops.append(-(live.pop((i, int(b["hf"][j]))) + 1))
            for k in range(int(ar[i]), int(ar[i + 1])):
                off = int(b["ref_out"][k])
                if off != int(FAIL):
                    live[(i, off)] = nslot
                    nslot += 1
                    ops.append(int(b["hs"][k]))
    return np.asarray(ops, dtype=np.int64)


def cuda_allocator_comparison(batches, alloc, flush, stream, max_ops: int = 60_000) -> dict:
    """The same operations through cudaMalloc/cudaFree and cudaMallocAsync/
    cudaFreeAsync (host-timed per call), beside this allocator on the same
    batches (device-timed per batch).  Sample: the longest prefix of the trace
    whose served allocations plus applied frees stay within ``max_ops``."""
    import torch

    from paper_2405_07079_gb300 import cuda_replay

    nb, served = 0, 0
    for b in batches:
        f, st, s, o = b["host"]
        k = int((st == 0).sum()) + int((o != FAIL).sum())
        if nb and served + k > max_ops:
            break
        nb += 1; served += k
    ops = cuda_replay.trace_ops(b["host"] for b in batches[:nb])
    res = {"sample": f"batches 0..{nb - 1} of the trace from an empty arena: their applied frees and "
                     f"served allocations in batch order ({ops.size} ops); failed allocations and "
                     "rejected frees are not replayed", "unit": UNIT}
    sptr = int(stream.cuda_stream)
    for mode in ("cudaMalloc", "cudaMallocAsync"):
        torch.cuda.synchronize()
        res[mode] = cuda_replay.replay(ops, mode, sptr)
    alloc.reset()
    ms = []
    for b in batches[:nb]:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        alloc.step(b["f"] if b["nf"] else None, b["s"] if b["na"] else None, out=b["out"], status=b["st"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = sum(ms) / 1e3
    reqs = sum(b["ops"] for b in batches[:nb])
    res["this_allocator"] = {"value": ops.size / t, "unit": UNIT, "ops": int(ops.size), "requests": reqs,
                             "requests_per_s": reqs / t, "ms_per_batch": 1e3 * t / nb,
                             "note": "device time of the batches that served these ops, failed requests included"}
    res["ratio_vs_cudaMalloc"] = res["this_allocator"]["value"] / res["cudaMalloc"]["value"]
    res["ratio_vs_cudaMallocAsync"] = res["this_allocator"]["value"] / res["cudaMallocAsync"]["value"]
    return res


E2E_DEPTH = 3  # host-buffer steps in flight in the pipelined end-to-end run


def e2e_host_calls(alloc, batches, steps, sptr, pipelined):
    """Replay ``steps`` batches of the trace through the host-buffer entry
    points (pinned inputs; copies, batch and result copy inside the call),
    from a fresh state, timed on the host.  Pipelined: hba_step_host_async
    with E2E_DEPTH output buffers in turn, the host waiting for and reading
    step k's first offset before issuing step k + E2E_DEPTH - 1.  Otherwise
    hba_step_host, which waits every step.  Returns (seconds, ops, H2D bytes,
    D2H bytes)."""
    import torch

    from paper_2405_07079_gb300 import hba_step_host, hba_step_host_async
    from paper_2405_07079_gb300.hba import _ptr

    nb = len(batches)
    stream = torch.cuda.current_stream()
    depth = E2E_DEPTH if pipelined else 1
    houts = [torch.empty(max(1, max(b["na"] for b in batches)), dtype=torch.int64).pin_memory()
             for _ in range(depth)]
    done = [torch.cuda.Event() for _ in range(depth)]
    alloc.reset()
    torch.cuda.synchronize()
    n_ops = h2d = d2h = 0
    seen = 0
    pos = 0
    t0 = time.perf_counter()
    for k in range(steps):
        if pos == nb:
            alloc.reset(); pos = 0
        b = batches[pos]; pos += 1
        j = k % depth
        if pipelined:
            if k >= depth - 1:
                i = (k - depth + 1) % depth
                done[i].synchronize()
                seen ^= int(houts[i][0])
            hba_step_host_async(alloc.h, _ptr(b["hf"]), b["nf"], 0, _ptr(b["hs"]), b["na"], _ptr(houts[j]), sptr)
            done[j].record(stream)
        else:
            hba_step_host(alloc.h, _ptr(b["hf"]), b["nf"], 0, _ptr(b["hs"]), b["na"], _ptr(houts[j]), sptr)
            seen ^= int(houts[j][0])
        n_ops += b["ops"]; h2d += 8 * (b["nf"] + b["na"]); d2h += 8 * b["na"]
    stream.synchronize()
    elapsed = time.perf_counter() - t0
    return elapsed, n_ops, h2d, d2h


def multi_e2e(ma, batches, steps, sptr):
    """The batched form end to end through the public host-buffer entry
    point: ``steps`` batches (wrapping with a reset) from pinned host
    buffers through hba_multi_step_host_async, E2E_DEPTH calls in flight, the
    host waiting for and reading step k's first offset before it issues step
    k + E2E_DEPTH - 1.  Timed on the host, copies and read-back included.
    Returns (seconds, ops, H2D bytes, D2H bytes)."""
    import torch

    from paper_2405_07079_gb300 import hba_multi_step_host_async, hba_reset

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    nb = min(len(batches), steps)
    host = [(pin(b["hfrow"].view(np.int32)), pin(b["harow"].view(np.int32)), pin(b["hf"].view(np.int64)),
             pin(b["hs"].view(np.int64))) for b in batches[:nb]]
    na_max = max(b["na"] for b in batches[:nb])
    houts = [torch.empty(max(1, na_max), dtype=torch.int64).pin_memory() for _ in range(E2E_DEPTH)]
    done = [torch.cuda.Event() for _ in range(E2E_DEPTH)]
    stream = torch.cuda.current_stream()
    hba_reset(ma.h, sptr)
    torch.cuda.synchronize()
    n_ops = h2d = d2h = seen = pos = 0
    t0 = time.perf_counter()
    for k in range(steps):
        if pos == nb:
            hba_reset(ma.h, sptr)
            pos = 0
        b, (hfr, har, hf, hs) = batches[pos], host[pos]
        pos += 1
        j = k % E2E_DEPTH
        if k >= E2E_DEPTH - 1:
            i = (k - E2E_DEPTH + 1) % E2E_DEPTH
            done[i].synchronize()
            seen ^= int(houts[i][0])
        hba_multi_step_host_async(ma.h, hfr.data_ptr(), hf.data_ptr() if b["nf"] else 0, b["nf"], har.data_ptr(),
                                  hs.data_ptr() if b["na"] else 0, b["na"], houts[j].data_ptr() if b["na"] else 0,
                                  0, sptr)
        done[j].record(stream)
        n_ops += b["ops"]
        h2d += 8 * (b["nf"] + b["na"]) + 2 * hfr.numel() * 4
        d2h += 8 * b["na"]
    stream.synchronize()
    return time.perf_counter() - t0, n_ops, h2d, d2h


def l2_copy_peak(dev, mib=32, copies=20, reps=5) -> dict:
    """An L2 bandwidth ceiling measured here: ``copies`` back-to-back
    device-to-device copies of a ``mib`` MiB buffer into another (both
    resident in the 129 MB L2) between two CUDA events, best of ``reps``
    after warm-up; read + write bytes per second."""
    import torch

    n = mib << 20
    a = torch.empty(n, dtype=torch.uint8, device=dev).fill_(1)
    b = torch.empty(n, dtype=torch.uint8, device=dev)
    for _ in range(5):
        b.copy_(a)
    best = float("inf")
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(copies):
            b.copy_(a)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3 / copies)
    return {"gbs": 2 * n / best / 1e9, "how": f"{copies} back-to-back torch copy_ of a {mib} MiB device buffer into "
                                               f"another (both L2-resident) between two CUDA events, best of {reps} "
                                               "after 5 warm-up copies; read + write bytes"}


def plain_large_figure(dev, steps=None) -> dict:
    """The plain single-arena form on the large trace (one 16 GiB arena,
    batches of 65,536): recorded untimed, then one pass replayed with an L2
    flush between steps, as the plain bench mode times it."""
    import torch

    from paper_2405_07079_gb300 import Allocator, workloads

    wl = workloads.large()
    with Allocator(wl.arena, wl.min_block, threads=1024) as alloc:
        batches = record_trace(wl, alloc, dev)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream()
        alloc.reset()
        n = len(batches) if steps is None else min(steps, len(batches))
        ms, served = [], 0
        for b in batches[:n]:
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            alloc.step(b["f"] if b["nf"] else None, b["s"] if b["na"] else None, out=b["out"], status=b["st"])
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            f, stat, s_, o = b["host"]
            served += int((stat == 0).sum()) + int((o != FAIL).sum())
    t = sum(ms) / 1e3
    ops = sum(b["ops"] for b in batches[:n])
    return {"workload": wl.name + ": " + wl.note, "steps": n, "value": ops / t, "served_ops_per_s": served / t,
            "unit": UNIT, "ms_per_step": 1e3 * t / n,
            "form": "plain single arena: prep grid + engine kernel per batch (k_single<1024>)",
            "l2": "flushed between steps (256 MiB write, untimed)"}


def multi_kernel_name(policy, shape, n_arenas, n_sms, wpc=8) -> str:
    """The batch kernel a multi-arena launch of this shape runs (the
    library's own choice, restated)."""
    if policy in FIT_POLICIES:
        return "k_fits<256>"
    if policy == "bitmask":
        return "k_bitmask<256>"
    if isinstance(shape, str):
        return "k_multi"
    threads, ctas = shape[0], shape[1]
    tl = ", two-level lists" if policy == "tlsf" else ""
    if threads == 32:
        from paper_2405_07079_gb300.tune import WARP_ARENAS_PER_CTA_TLSF
        need = -(-n_arenas // (WARP_ARENAS_PER_CTA_TLSF if tl else wpc))
        grid = min(ctas, need) if ctas else need
        return f"k_prep + k_multi_warp<{2 if grid <= 2 * n_sms else 4}{tl}>"
    return f"k_prep + k_multi<{threads}{tl}>"


# The sources the batch engine's kernels (k_prep, k_single, k_multi,
# k_multi_warp, k_serve) are built from; the other policies' headers do not
# enter them.
ENGINE_SOURCES = ("paper_2405_07079_gb300/csrc/hba_engine.cuh", "paper_2405_07079_gb300/csrc/hba_capi.cu",
                  "paper_2405_07079_gb300/csrc/hba_serve.cuh", "include/hba.h")


def kernel_sources_digest() -> str:
    """A digest of the engine kernels' sources: DRAM traffic taken with ncu
    is quoted only while the kernels are the ones captured."""
    import hashlib

    h = hashlib.sha256()
    for path in (os.path.join(ROOT, p) for p in ENGINE_SOURCES):
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per step from an
# ncu capture, with the algorithmic bytes of the captured steps: keyed by the
# kernel-source digest it was taken on, and by the kernel.
PROFILED_TRAFFIC = {
    # profiles/k_multi_warp_batched4096.txt: the default batched command, 20 timed steps
    ("eed269d8444ba035", "k_prep + k_multi_warp<4>"): {"dram_bytes_per_step": 990.2e6,
                                                        "algorithmic_bytes_per_step": 804.75e6},
    # profiles/k_single_tiny_k_serve_l2.txt: the tiny trace, 6 timed launches; one 50 ms serving run
    ("eed269d8444ba035", "k_single<128>"): {"dram_bytes_per_step": 162.6e3, "algorithmic_bytes_per_step": 10.71e3},
    ("eed269d8444ba035", "k_serve"): {"dram_bytes_per_step": 6.747e6, "algorithmic_bytes_per_step": 14.27e6},
    # profiles/k_single_large16GiB.txt: the large trace, 30 timed steps, both kernels
    ("eed269d8444ba035", "k_prep + k_single<1024>"): {"dram_bytes_per_step": 559.5e3,
                                                       "algorithmic_bytes_per_step": 2.087e6},
}


def profiled_traffic(kernel: str, algorithmic_bytes_per_step: float):
    """DRAM traffic per step for this kernel from its ncu capture, scaled to
    this run's algorithmic bytes per step (traffic grows with the requests a
    step carries), or None when no capture of the current sources exists."""
    rec = PROFILED_TRAFFIC.get((kernel_sources_digest(), kernel))
    if rec is None:
        return None
    return rec["dram_bytes_per_step"] * algorithmic_bytes_per_step / rec["algorithmic_bytes_per_step"]


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2405_07079_gb300 import Allocator, workloads

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = {"large": workloads.large, "tiny": workloads.tiny, "frag": workloads.frag,
          "usage": workloads.usage, "objects": workloads.objects}[args.workload]()
    alloc = Allocator(wl.arena, wl.min_block, threads=args.threads, ctas=args.ctas, policy=args.policy)
    space = []
    batches = record_trace(wl, alloc, dev, space)
    nb = len(batches)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    sptr = int(stream.cuda_stream)

    def launch(b):
        alloc.step(b["f"] if b["nf"] else None, b["s"] if b["na"] else None, out=b["out"], status=b["st"])

    # replay: warm-up then timed steps (the trace wraps with an untimed reset)
    alloc.reset()
    pos = 0
    for _ in range(args.warmup):
        if pos == nb:
            alloc.reset(); pos = 0
        flush.zero_()
        launch(batches[pos]); pos += 1
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    idx = []
    launches = 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clocks, torch.cuda.nvtx.range("timed"):
        for k in range(args.steps):
            if pos == nb:
                alloc.reset(); pos = 0
            flush.zero_()
            c0 = alloc.launches()
            ev[k][0].record(stream)
            launch(batches[pos])
            ev[k][1].record(stream)
            launches += alloc.launches() - c0
            idx.append(pos); pos += 1
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    busy_s = sum(step_ms) / 1e3
    ops = sum(batches[i]["ops"] for i in idx)
    served = sum(batches[i]["served"] for i in idx)
    nbytes = sum(batches[i]["bytes"] for i in idx)

    # e2e through the public host-buffer entry points, from a fresh state
    e2e_s, e2e_ops, e2e_h2d, e2e_d2h = e2e_host_calls(alloc, batches, args.steps, sptr, pipelined=True)
    sync_s, sync_ops, _, _ = e2e_host_calls(alloc, batches, args.steps, sptr, pipelined=False)

    (busy_s, e2e_s, sync_s), (ops_all, e2e_all, sync_all, served_all) = reduce_over_ranks(
        [busy_s, e2e_s, sync_s], [ops, e2e_ops, sync_ops, served], world, dev)
    stats = alloc.stats()
    cuda_cmp = None
    if rank == 0 and not args.no_cuda_baseline:
        cuda_cmp = cuda_allocator_comparison(batches, alloc, flush, stream)
    alloc.close()
    if rank != 0:
        return None
    peak, peak_src = _peaks()
    # one launch a step where the engine gathers its own frees (small batches)
    eng = f"k_single<{alloc_threads(args)}" + (", two-level lists>" if args.policy == "tlsf" else ">")
    plain_kernel = eng if launches <= args.steps else "k_prep + " + eng
    bound, peak_note = "hbm", f"{peak_src} hbm_gbs"
    if wl.arena // wl.min_block * 16 <= 32 << 20:  # a record table that stays in L2
        l2 = l2_copy_peak(dev)
        bound, peak, peak_note = "l2", l2["gbs"], "measured here: " + l2["how"]
    achieved_gbs = nbytes / busy_s / 1e9
    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": ops_all / busy_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * busy_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "served_ops_per_s": served_all / busy_s,
        "config": {"workload": wl.name + ": " + wl.note, "policy": args.policy, "parallelism": f"replicas x{world}",
                   "form": ("two-level segregated fit through the batch engine (512 lists: first level in the "
                            "bitmap word, second level in shared memory)"
                            if args.policy == "tlsf" else
                            f"{args.policy} fit on address-sorted lists: one CTA applies the batch (k_fits<256>)"
                            if args.policy in FIT_POLICIES else
                            "bitmask pool: one CTA applies the batch, bitmaps in shared memory (k_bitmask<256>)"
                            if args.policy == "bitmask" else
                            "plain single arena: one thread-block cluster per batch (engine CTA + CTAs that "
                            "gather the frees' records into its shared memory and pre-fill failures)"
                            if args.ctas >= 2 else "plain single arena: prep grid + engine kernel per batch"),
                   "threads_per_cta": (256 if args.policy in FIT_POLICIES + ("bitmask",)
                                       else alloc_threads(args)),
                   "l2": "flushed between steps (256 MiB write, untimed)", "trace_batches": nb,
                   "ops_per_step_mean": ops / max(1, args.steps)},
        "roofline": {"bound": bound, "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                     "frac": achieved_gbs / peak,
                     "traffic": (profiled_traffic(plain_kernel, nbytes / max(1, args.steps))
                                 if args.ctas < 2 and args.policy in ("segfit", "tlsf") else None),
                     "peak_source": peak_note,
                     "kernel": ("k_fits<256>" if args.policy in FIT_POLICIES else
                                "k_bitmask<256>" if args.policy == "bitmask" else
                                f"k_single_cl<{alloc_threads(args)}>" if args.ctas >= 2
                                else plain_kernel),
                     "bytes_model": "168 B per served alloc, 16 B per failed alloc, 216 B per applied free, 9 B per rejected free"},
        "latency_us": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "unit": "per batch of one step"},
        "e2e": {"value": e2e_all / e2e_s, "unit": UNIT, "h2d_bytes_per_step": e2e_h2d // max(1, args.steps),
                "d2h_bytes_per_step": e2e_d2h // max(1, args.steps), "api": "hba_step_host_async",
                "form": (f"{E2E_DEPTH} steps in flight; each step's offsets are read on the host "
                         f"{E2E_DEPTH - 1} steps later; no L2 flush between steps"),
                "synchronous": {"value": sync_all / sync_s, "unit": UNIT, "api": "hba_step_host",
                                "form": "one host wait per step"}},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "final_stats": {k: stats[k] for k in ("alloc_ok", "alloc_fail", "free_ok", "free_fail")},
        "memory_usage": space_report(space, alloc.arena_bytes),
    }
    if cuda_cmp is not None:
        line["cuda_allocators"] = cuda_cmp
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.policy)
    return line


def run_multi(args, rank, world, local_rank):
    """The batched form: thousands of independent arenas, one batch of all of
    them per step (prep grid + one multi-arena launch)."""
    import torch

    from paper_2405_07079_gb300 import Allocator, MultiAllocator, hba_step, workloads
    from paper_2405_07079_gb300.hba import _ptr
    from paper_2405_07079_gb300.tune import autotune_multi

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    A = workloads.multi_arena_sizes(args.arenas, lo=args.arena_min << 20, hi=args.arena_max << 20)
    gen = workloads.MultiLifetimes(A, n_batches=args.batches)
    cap = args.arenas * 2048 + 1
    ma = MultiAllocator(A, 256, max_total_frees=cap, policy=args.policy, max_total_allocs=cap)
    t_rec = time.time()
    batches = []
    while (b := gen.next_batch()) is not None:
        frow, f, arow, s = b
        d = {"frow": torch.from_numpy(frow.view(np.int32)).to(dev), "f": torch.from_numpy(f.view(np.int64)).to(dev),
             "arow": torch.from_numpy(arow.view(np.int32)).to(dev), "s": torch.from_numpy(s.view(np.int64)).to(dev),
             "nf": f.size, "na": s.size, "ops": f.size + s.size, "hfrow": frow, "harow": arow, "hf": f, "hs": s}
        d["out"] = torch.empty(s.size, dtype=torch.int64, device=dev)
        d["st"] = torch.empty(f.size, dtype=torch.uint8, device=dev)
        ma.step(d["frow"], d["f"], d["arow"], d["s"], d["out"], d["st"])
        o = d["out"].cpu().numpy().view(np.uint64)
        gen.feed(o)
        stat = d["st"].cpu().numpy()
        n_ok, n_fok = int((o != FAIL).sum()), int((stat == 0).sum())
        d["bytes"] = (BYTES_ALLOC_OK * n_ok + BYTES_ALLOC_FAIL * (s.size - n_ok)
                      + BYTES_FREE_OK * n_fok + BYTES_FREE_REJECTED * (f.size - n_fok))
        d["served"] = n_ok + n_fok
        d["ref_out"] = o.copy()
        d["ref_st"] = stat.copy()
        batches.append(d)
    t_rec = time.time() - t_rec
    if args.policy in FIT_POLICIES:
        best, table = f"one CTA per arena ({args.policy} fit)", {}
    elif args.shape:
        best = tuple(int(x) for x in args.shape.split(","))
        ma.set_shape(*best)
        table = {}
    else:
        best, table = autotune_multi(ma, batches, n_probe=3)
    nb = len(batches)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def launch(b):
        ma.step(b["frow"], b["f"], b["arow"], b["s"], b["out"], b["st"], stream=stream)

    ma_reset = lambda: __import__("paper_2405_07079_gb300").hba_reset(ma.h, int(stream.cuda_stream))
    ma_reset()
    pos = 0
    for _ in range(args.warmup):
        if pos == nb:
            ma_reset(); pos = 0
        flush.zero_()
        launch(batches[pos]); pos += 1
    steps = args.steps if args.steps else nb
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    idx = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    from paper_2405_07079_gb300 import hba_launch_count
    launches0 = hba_launch_count(ma.h)
    with ClockSampler(local_rank) as clocks, torch.cuda.nvtx.range("timed"):
        for k in range(steps):
            if pos == nb:
                ma_reset(); pos = 0
            flush.zero_()
            ev[k][0].record(stream)
            launch(batches[pos])
            ev[k][1].record(stream)
            idx.append(pos); pos += 1
        torch.cuda.synchronize()
    launches = hba_launch_count(ma.h) - launches0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    busy_s = sum(step_ms) / 1e3
    ops = sum(batches[i]["ops"] for i in idx)
    served = sum(batches[i]["served"] for i in idx)
    nbytes = sum(batches[i]["bytes"] for i in idx)
    # e2e through the public host-buffer entry point, from a fresh state
    sptr = int(stream.cuda_stream)
    e2e_s, e2e_ops, e2e_h2d, e2e_d2h = multi_e2e(ma, batches, steps, sptr)
    (busy_all, e2e_all_s), (ops_all, served_all, e2e_all) = reduce_over_ranks(
        [busy_s, e2e_s], [ops, served, e2e_ops], world, dev)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    # the plain form on the same requests: the first P arenas, one handle and
    # one launch per arena per batch; results must equal the batched form's
    P = min(args.plain_arenas, args.arenas)
    plain = [Allocator(int(A[i]), 256, max_batch=2048, policy=args.policy) for i in range(P)]
    plain_ops, plain_ms, nb_plain = 0, 0.0, min(nb, 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for bi in range(nb_plain):
        b = batches[bi]
        outs = []
        e0.record(stream)
        for i in range(P):
            f0, f1, a0, a1 = int(b["hfrow"][i]), int(b["hfrow"][i + 1]), int(b["harow"][i]), int(b["harow"][i + 1])
            o = b["out"][a0:a1]
            hba_step(plain[i].h, _ptr(b["f"][f0:f1]), f1 - f0, 0, _ptr(b["s"][a0:a1]), a1 - a0, _ptr(o),
                     int(stream.cuda_stream))
            plain_ops += (f1 - f0) + (a1 - a0)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms += e0.elapsed_time(e1)
        got = b["out"][: int(b["harow"][P])].cpu().numpy().view(np.uint64)
        if not np.array_equal(got, b["ref_out"][: int(b["harow"][P])]):
            raise AssertionError(f"plain form differs from the batched form in batch {bi}")
    for a in plain:
        a.close()
    ma.close()
    large = plain_large_figure(dev) if args.policy == "segfit" and not args.no_plain_large else None
    if rank != 0:
        return None
    extra = {}
    if not args.no_cpu_baseline:
        # the oracle on the first arenas, whole sequences, sharded over the host cores
        K = min(args.oracle_arenas, args.arenas)
        seqs = [[(b["hf"][int(b["hfrow"][i]):int(b["hfrow"][i + 1])], b["hs"][int(b["harow"][i]):int(b["harow"][i + 1])])
                 for b in batches] for i in range(K)]
        v, cores, res = oracle_pool_baseline(A[:K], 256, seqs, policy=args.policy)
        for i in range(K):
            for bi, b in enumerate(batches):
                a0, a1 = int(b["harow"][i]), int(b["harow"][i + 1])
                if not np.array_equal(res[i][bi][0], b["ref_out"][a0:a1]):
                    raise AssertionError(f"oracle and batched form differ: arena {i}, batch {bi}")
        extra["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"the first {K} arenas, all {nb} batches, sharded over {cores} "
                                           "spawned processes; wall time of the pool (results equal the GPU's)"}
    if not args.no_cuda_baseline:
        from paper_2405_07079_gb300 import cuda_replay
        ops_l = cuda_replay_ops_multi(batches[:nb_plain], range(P))
        sptr = int(stream.cuda_stream)
        extra["cuda_allocators"] = {"sample": f"the plain-form comparison's requests (first {P} arenas, "
                                              f"{nb_plain} batches): applied frees and served allocations "
                                              f"({ops_l.size} ops)", "unit": UNIT}
        for mode in ("cudaMalloc", "cudaMallocAsync"):
            torch.cuda.synchronize()
            extra["cuda_allocators"][mode] = cuda_replay.replay(ops_l, mode, sptr)
    peak, peak_src = _peaks()
    achieved = nbytes / busy_s / 1e9
    lat = sorted(step_ms)
    kernel = multi_kernel_name(args.policy, best, args.arenas, n_sms)
    plain_v = plain_ops / (plain_ms / 1e3)
    line = {
        "metric": METRIC, "value": ops_all / busy_all, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * busy_all / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "served_ops_per_s": served_all / busy_all,
        "config": {"policy": args.policy,
                   "workload": f"batched-{args.arenas}: {args.arenas} arenas log-uniform "
                               f"{args.arena_min} MiB-{args.arena_max} MiB, min block 256 B, U{{0..2048}} requests "
                               f"per arena per batch, {nb} batches",
                   "form": ("batched: one launch per batch, one CTA per arena (k_fits<256>)"
                            if args.policy in FIT_POLICIES
                            else "batched: one launch per batch, one CTA per pool (k_bitmask<256>)"
                            if args.policy == "bitmask"
                            else "batched: prep grid + one multi-arena launch per batch"),
                   "parallelism": f"replicas x{world}",
                   "shape": (best if isinstance(best, str) else
                             {"threads": best[0], "ctas": best[1], "smem_bytes": best[2]}),
                   "l2": "flushed between steps (256 MiB write, untimed); the record tables (about 87 GB) "
                         "are far larger than L2", "ops_per_step_mean": ops / steps,
                   "record_s": round(t_rec, 1)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": profiled_traffic(kernel, nbytes / steps), "peak_source": f"{peak_src} hbm_gbs",
                     "kernel": kernel,
                     "timed": "CUDA events around each step's launches (the prep grid and the batch kernel)",
                     "bytes_model": "168 B per served alloc, 16 B per failed alloc, 216 B per applied free, 9 B per rejected free"},
        "latency_us": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "unit": "per batch of all arenas"},
        "e2e": {"value": e2e_all / e2e_all_s, "unit": UNIT, "h2d_bytes_per_step": e2e_h2d // max(1, steps),
                "d2h_bytes_per_step": e2e_d2h // max(1, steps), "api": "hba_multi_step_host_async",
                "form": (f"pinned host buffers; {E2E_DEPTH} steps in flight; each step's offsets are read on the "
                         f"host {E2E_DEPTH - 1} steps later; no L2 flush between steps")},
        "plain_form_same_requests": {"arenas": P, "batches": nb_plain, "value": plain_v, "unit": UNIT,
                                     "form": "one handle and one hba_step launch per arena per batch",
                                     "results_equal": True},
        "batched_over_plain": (ops_all / busy_all) / plain_v,
        "autotune_ms": {f"t{t}_c{c}_s{m}": round(v, 3) for (t, c, m), v in sorted(table.items())},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    if large is not None:
        line["plain_single_arena_large"] = large
        line["batched_over_plain_large"] = (ops_all / busy_all) / large["value"]
    line.update(extra)
    return line


def run_serve(args, rank, world, local_rank):
    """The serving form: one 80 GiB arena of 16 KiB pages, Poisson arrivals
    (sweep of rates), malloc of U{1..512} pages held Exp(20 ms), admission by
    free memory with a 1M-deep queue; the loop runs on the device."""
    import torch

    from paper_2405_07079_gb300 import Allocator, hba_step, log_batches, serve, workloads
    from paper_2405_07079_gb300.hba import _ptr

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    arena, page = 80 << 30, 16 << 10
    sweep = []
    kept = [None, None]  # the first rate's run and the fastest later one, for the plain replay
    lams = [float(x) * 1e6 for x in args.lams.split(",")]
    for li, lam in enumerate(lams):
        arr = workloads.serving_arrivals(lam, args.serve_seconds)
        with Allocator(arena, page, threads=256) as a:
            served, log, rep = serve(a, arr)
        adm = served[:, 0] != np.uint64(0xFFFFFFFFFFFFFFFE)
        lat = (served[adm, 1] - arr[adm, 0]).astype(np.float64) / 1e3
        ops = rep["alloc_ok"] + rep["alloc_fail"] + rep["frees"]
        sec = max(rep["elapsed_ns"], 1) / 1e9
        sweep.append({"lambda_req_s": lam, "arrivals": rep["arrivals"], "admitted": rep["admitted"],
                      "rejected": rep["rejected"], "alloc_ok": rep["alloc_ok"], "alloc_fail": rep["alloc_fail"],
                      "frees": rep["frees"], "ticks": rep["ticks"], "max_queue": rep["max_queue"],
                      "elapsed_s": sec, "ops_per_s": ops / sec, "admitted_per_s": rep["admitted"] / sec,
                      "p50_us": float(np.percentile(lat, 50)) if lat.size else None,
                      "p99_us": float(np.percentile(lat, 99)) if lat.size else None, "status": rep["status"]})
        keep = li == 0 or sweep[-1]["ops_per_s"] >= max(r["ops_per_s"] for r in sweep)
        if keep:
            kept[0 if li == 0 else 1] = (lam, arr, served, log, ops)

    def plain_replay(lam, arr, served, log, ops):
        """The plain form on the same batches: one launch pair per logged tick,
        back to back from the host; results must equal the serving loop's."""
        dt = []
        for fid, aid in log_batches(log):
            f = torch.from_numpy(served[fid, 0].view(np.int64)).to(dev)
            s_ = torch.from_numpy(arr[aid, 1].view(np.int64)).to(dev)
            dt.append((f, s_, torch.empty(max(aid.size, 1), dtype=torch.int64, device=dev), aid))
        stream = torch.cuda.current_stream()
        with Allocator(arena, page, threads=256) as pa:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for f, s_, o, aid in dt:
                hba_step(pa.h, _ptr(f), f.numel(), 0, _ptr(s_), s_.numel(), _ptr(o), int(stream.cuda_stream))
            e1.record(stream)
            torch.cuda.synchronize()
            pms = e0.elapsed_time(e1)
            equal = all(np.array_equal(o[:aid.size].cpu().numpy().view(np.uint64), served[aid, 0]) for f, s_, o, aid in dt)
        return {"lambda_req_s": lam, "ticks": len(dt), "ops_per_s": ops / (pms / 1e3), "elapsed_s": pms / 1e3,
                "results_equal": bool(equal)}

    plain = [plain_replay(*k) for k in kept if k is not None]
    extra = {}
    lam0, arr0, served0, log0, ops0 = kept[0]
    ticks0 = log_batches(log0)
    if not args.no_cpu_baseline and rank == 0:
        # the oracle on the first rate's ticks, one host core
        import oracle
        oracle.build()
        o = oracle.Oracle(arena, page)
        t_or, n_or = 0.0, 0
        for fid, aid in ticks0:
            f, s_ = served0[fid, 0].copy(), arr0[aid, 1].copy()
            t0 = time.perf_counter()
            out, _ = o.batch(f, s_)
            t_or += time.perf_counter() - t0
            n_or += f.size + s_.size
            if not np.array_equal(out, served0[aid, 0]):
                raise AssertionError("oracle and serving loop differ")
        extra["cpu_baseline"] = {"value": n_or / t_or, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"the {len(ticks0)} ticks of the {lam0 / 1e6:g} M req/s run, replayed in "
                                           "order (results equal the serving loop's); oracle calls timed"}
    if not args.no_cuda_baseline and rank == 0:
        from paper_2405_07079_gb300 import cuda_replay
        live, ops_l, nslot = {}, [], 0
        for fid, aid in ticks0:
            for off in served0[fid, 0].tolist():
                ops_l.append(-(live.pop(off) + 1))
            for sz, off in zip(arr0[aid, 1].tolist(), served0[aid, 0].tolist()):
                if off != int(FAIL):
                    live[off] = nslot
                    nslot += 1
                    ops_l.append(int(sz))
        ops_l = np.asarray(ops_l, dtype=np.int64)
        sptr = int(torch.cuda.current_stream().cuda_stream)
        extra["cuda_allocators"] = {"sample": f"the {lam0 / 1e6:g} M req/s run's served allocations and frees in "
                                              f"tick order ({ops_l.size} ops)", "unit": UNIT}
        for mode in ("cudaMalloc", "cudaMallocAsync"):
            torch.cuda.synchronize()
            extra["cuda_allocators"][mode] = cuda_replay.replay(ops_l, mode, sptr)
    best = max(sweep, key=lambda r: r["ops_per_s"])
    l2 = l2_copy_peak(dev)
    b_alg = (BYTES_ALLOC_OK * best["alloc_ok"] + BYTES_ALLOC_FAIL * best["alloc_fail"]
             + BYTES_FREE_OK * best["frees"])
    roof = {"bound": "l2", "achieved": b_alg / best["elapsed_s"] / 1e9, "peak": l2["gbs"], "unit": "GB/s",
            "frac": b_alg / best["elapsed_s"] / 1e9 / l2["gbs"], "traffic": profiled_traffic("k_serve", b_alg),
            "peak_source": "measured here: " + l2["how"], "kernel": "k_serve",
            "at_lambda": best["lambda_req_s"],
            "note": "the 80 GiB arena's record table (84 MB) and list heads fit in L2",
            "bytes_model": "168 B per served alloc, 16 B per failed alloc, 216 B per applied free"}
    (sec_all,), (ops_all,) = reduce_over_ranks([best["elapsed_s"]], [best["ops_per_s"] * best["elapsed_s"]], world,
                                               torch.device("cuda", local_rank))
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": ops_all / sec_all, "unit": UNIT, "n_gpus": world, "steps": len(sweep),
        "warmup": 0, "ms_per_step": 1e3 * sec_all, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"serving: 80 GiB arena of 16 KiB pages, Poisson arrivals {args.lams} M req/s for "
                               f"{args.serve_seconds} s each, U{{1..512}} pages held Exp(20 ms), queue 1M",
                   "form": "serving loop: one persistent CTA, device-resident queue and timing wheel",
                   "parallelism": f"replicas x{world}"},
        "latency_us": {"p50": best["p50_us"], "p99": best["p99_us"], "unit": "arrival to result, admitted requests",
                       "at_lambda": best["lambda_req_s"]},
        "roofline": roof,
        "sweep": sweep, "plain_form_same_batches": plain,
        "serving_over_plain_at_best": (best["ops_per_s"] / plain[-1]["ops_per_s"]
                                       if plain and plain[-1]["lambda_req_s"] == best["lambda_req_s"] else None),
        "gpu_launches": len(sweep),
        **extra,
    }


def alloc_threads(args):
    """CTA width of the plain form: --threads, else the library's choice by
    batch size (1,024 for the large and frag batches, 128 for the tiny ones
    and the one-op batches of the memory-usage workload)."""
    if args.threads:
        return args.threads
    return 128 if args.workload in ("tiny", "usage", "objects") else 1024


def oracle_steps(wl, n_steps=None, warmup=0, policy="segfit"):
    """Closed-loop client + oracle.  The first ``warmup`` batches run untimed;
    returns (oracle seconds, ops, timed steps) over the next ``n_steps``
    batches (None: to the end of the trace).  The trace restarts from a fresh
    oracle when it ends."""
    import oracle

    o = _make_oracle(oracle, wl.arena, wl.min_block, policy)
    client = wl.make()
    t_or, ops, k, seen = 0.0, 0, 0, 0
    while n_steps is None or k < n_steps:
        b = client.next_batch()
        if b is None:
            if n_steps is None:
                break
            o = _make_oracle(oracle, wl.arena, wl.min_block, policy)
            client = wl.make()
            continue
        t0 = time.perf_counter()
        out, _ = o.batch(*b)
        dt = time.perf_counter() - t0
        client.feed(out)
        seen += 1
        if seen > warmup:
            t_or += dt
            ops += b[0].size + b[1].size
            k += 1
    return t_or, ops, k


def cpu_baseline(wl, policy="segfit") -> dict:
    t, ops, k = oracle_steps(wl, policy=policy)
    return {"value": ops / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the whole trace ({k} batches, {ops} ops), closed loop, single thread; "
                      f"oracle calls timed ({t:.3f} s)"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    if args.workload == "multi":
        return run_reference_multi(args, world)
    if args.workload == "serve":
        return {"impl": "reference", "unavailable": "the serving loop has no oracle arm: its oracle replays the "
                                                    "device's tick log, which needs the GPU run first"}
    from paper_2405_07079_gb300 import workloads

    steps = 1530 if args.steps is None else args.steps
    wl = {"large": workloads.large, "tiny": workloads.tiny, "frag": workloads.frag,
          "usage": workloads.usage, "objects": workloads.objects}[args.workload]()
    t, ops, k = oracle_steps(wl, n_steps=steps, warmup=args.warmup, policy=args.policy)
    v = ops / t
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": wl.name + ": " + wl.note, "policy": args.policy,
                       "parallelism": "single host thread",
                       "form": "sequential CPU oracle, one batch per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"batches {args.warmup}..{args.warmup + steps - 1} of the trace "
                                       "(wrapping to a fresh oracle), oracle calls timed"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_multi(args, world):
    """The oracle arm of the batched form: the same 4,096-arena workload,
    one oracle per arena, closed loop; a step is one batch of every arena,
    applied arena by arena on one host thread (oracle calls timed)."""
    import oracle
    from paper_2405_07079_gb300 import workloads

    oracle.build()
    A = workloads.multi_arena_sizes(args.arenas, lo=args.arena_min << 20, hi=args.arena_max << 20)
    steps = 20 if not args.steps else args.steps
    gen = workloads.MultiLifetimes(A, n_batches=args.warmup + steps)
    orcs = [_make_oracle(oracle, int(a), 256, args.policy) for a in A]
    t_or, ops, k = 0.0, 0, 0
    while (b := gen.next_batch()) is not None:
        frow, f, arow, s = b
        outs = []
        dt = 0.0
        for i in range(A.size):
            fi, si = f[frow[i]:frow[i + 1]], s[arow[i]:arow[i + 1]]
            t0 = time.perf_counter()
            o, _ = orcs[i].batch(fi, si)
            dt += time.perf_counter() - t0
            outs.append(o)
        gen.feed(np.concatenate(outs))
        k += 1
        if k > args.warmup:
            t_or += dt
            ops += f.size + s.size
    v = ops / t_or
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_or / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"policy": args.policy,
                       "workload": f"batched-{args.arenas}: {args.arenas} arenas log-uniform 64 MiB-1 GiB, "
                                   f"min block 256 B, U{{0..2048}} requests per arena per batch",
                       "parallelism": "single host thread",
                       "form": "sequential CPU oracle per arena, one batch of all arenas per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"batches {args.warmup}..{args.warmup + steps - 1} of the batched trace "
                                       f"({ops} requests), every arena; each arena's oracle call timed"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: one pass over the recorded batches for the batched form, "
                         "1,530 = ten passes over the large trace for the plain form)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=["large", "tiny", "frag", "usage", "objects", "multi", "serve"],
                    default="multi",
                    help="multi (default): the batched form, 4,096 arenas in one launch per batch; large, tiny, "
                         "frag, usage, objects: the plain single-arena form; serve: the serving loop")
    ap.add_argument("--policy", choices=["segfit", "tlsf", "first", "next", "best", "bitmask"], default="segfit",
                    help="segregated fit (§5.1), two-level segregated fit (§5.2), a sequential fit on "
                         "address-sorted lists (§4), or the bitmask pool (§3.2); the serving loop is segfit only")
    ap.add_argument("--lams", default="1,2,5,10,20,50")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--arenas", type=int, default=4096)
    ap.add_argument("--batches", type=int, default=200)
    ap.add_argument("--arena-min", type=int, default=64, help="batched form: smallest arena, MiB")
    ap.add_argument("--arena-max", type=int, default=1024, help="batched form: largest arena, MiB")
    ap.add_argument("--plain-arenas", type=int, default=64)
    ap.add_argument("--oracle-arenas", type=int, default=256,
                    help="batched form: arenas the oracle baseline runs (whole sequences)")
    ap.add_argument("--shape", default="",
                    help="batched form: threads,ctas,smem_bytes instead of autotuning")
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--ctas", type=int, default=0,
                    help="single arena: batch cluster size (0 or 1 = prep grid + engine; 2..8 = engine CTA + gathering CTAs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cuda-baseline", action="store_true")
    ap.add_argument("--no-plain-large", action="store_true",
                    help="batched form: skip the plain single-arena large-trace figure")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        if args.workload == "serve":
            if args.policy != "segfit":
                ap.error("the serving loop runs segregated fit only")
            line = run_serve(args, rank, world, local_rank)
        elif args.workload == "multi":
            if args.steps is None:
                args.steps = 0  # one pass over the recorded batches
            line = run_multi(args, rank, world, local_rank)
        else:
            if args.steps is None:
                args.steps = 1530
            line = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
