// Allocation-free variant of the FP32 forward filter.
//
// Some callers cannot allocate device memory at the moment they need the
// filter: a real-time audio callback that must not block on the CUDA
// allocator, a plugin running inside a host application that owns the GPU
// memory budget, or code that runs between pre-planned allocations.  For
// them this file provides lp_tv_forward_noalloc_f32, which takes inputs and
// outputs like lp_tv_forward_f32 but keeps the scan's scratch data (chunk
// maps and chunk states) in a fixed array compiled into the library instead
// of a caller-supplied workspace.
#include <stdint.h>

#include <atomic>

#include <cuda_runtime.h>

#include "tvlp.h"

// The scratch array.  Every GPU that loads the library holds it until the
// process exits.  All calls share it and each call overwrites what the
// previous one left; nothing in it needs to start at zero.
static __device__ __align__(256) unsigned char g_tvlp_noalloc_scratch[LP_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDev = 64;

// Device address of the scratch array on the current device; looked up once
// per device (the host-side symbol is not a device address).  Two host
// threads making their first call on a device at the same time both look it
// up and store the same address: the cache entries are atomics.
void *scratch_address() {
    static std::atomic<void *> cached[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return nullptr;
    }
    void *ptr = cached[dev].load(std::memory_order_relaxed);
    if (ptr == nullptr) {
        if (cudaGetSymbolAddress(&ptr, g_tvlp_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        cached[dev].store(ptr, std::memory_order_relaxed);
    }
    return ptr;
}

}  // namespace

extern "C" int lp_tv_forward_noalloc_f32(int B, int64_t T, int M, const float *a, const float *e, const float *zi,
                                         float *s, void *stream) {
    if (B < 0 || T < 0 || M < 0) return LP_EINVAL;
    if (B == 0 || T == 0) return LP_OK;
    // the chunked scan needs lp_tv_workspace_bytes(...) of scratch; refuse
    // problems whose scratch does not fit the fixed array
    const size_t need = lp_tv_workspace_bytes(B, T, M, 0, LP_DTYPE_F32);
    if (M > 0 && need == 0) return LP_EUNSUPPORTED;
    if (need > (size_t)LP_NOALLOC_SCRATCH_BYTES) return LP_ETOOBIG;
    void *scratch = M > 0 ? scratch_address() : nullptr;
    if (M > 0 && scratch == nullptr) return LP_ECUDA;
    return lp_tv_forward_f32(B, T, M, a, e, zi, s, nullptr, 0, LP_ALGO_CHUNKED, scratch,
                             (size_t)LP_NOALLOC_SCRATCH_BYTES, stream);
}
