// Replays an allocation trace through the CUDA runtime's own allocators, as
// the comparison the paper draws (§6: segregated fit against cudaMalloc and
// cudaFree on the same operation order).  Host code only; no kernels.
//
// Trace encoding, one int64 per operation, in order:
//   op >= 0        malloc of `op` bytes; the k-th malloc of the trace fills slot k
//   op <  0        free of slot (-op - 1)
// mode 0: cudaMalloc / cudaFree.  mode 1: cudaMallocAsync / cudaFreeAsync on
// `stream` with the device's default memory pool.
//
// lat_ns[i] (optional) receives the host wall time of operation i; the return
// value is the total wall time in ns including a final synchronisation (so the
// asynchronous mode pays for its queued work), or a negative CUDA error code.
// Slots that are still live at the end are released outside the timed region.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <vector>

namespace {

inline int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

extern "C" int64_t car_replay(const int64_t* ops, int64_t n, int mode, int64_t* lat_ns, void* stream) {
    if (n < 0 || (n > 0 && !ops) || (mode != 0 && mode != 1)) return -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t nslots = 0;
    for (int64_t i = 0; i < n; ++i) nslots += ops[i] >= 0;
    std::vector<void*> slot(static_cast<size_t>(nslots), nullptr);
    int64_t next = 0;
    cudaError_t err = cudaSuccess;
    const int64_t t0 = now_ns();
    for (int64_t i = 0; i < n && err == cudaSuccess; ++i) {
        const int64_t t = lat_ns ? now_ns() : 0;
        const int64_t op = ops[i];
        if (op >= 0) {
            void* p = nullptr;
            err = mode == 0 ? cudaMalloc(&p, static_cast<size_t>(op))
                            : cudaMallocAsync(&p, static_cast<size_t>(op), s);
            slot[static_cast<size_t>(next++)] = p;
        } else {
            const int64_t k = -op - 1;
            if (k >= next || !slot[static_cast<size_t>(k)]) return -2;  // free of an unknown slot
            err = mode == 0 ? cudaFree(slot[static_cast<size_t>(k)])
                            : cudaFreeAsync(slot[static_cast<size_t>(k)], s);
            slot[static_cast<size_t>(k)] = nullptr;
        }
        if (lat_ns) lat_ns[i] = now_ns() - t;
    }
    if (err == cudaSuccess) err = mode == 0 ? cudaDeviceSynchronize() : cudaStreamSynchronize(s);
    const int64_t total = now_ns() - t0;
    for (void* p : slot)
        if (p) {
            if (mode == 0) cudaFree(p);
            else cudaFreeAsync(p, s);
        }
    if (mode == 1) cudaStreamSynchronize(s);
    return err == cudaSuccess ? total : -static_cast<int64_t>(err) - 1000;
}
