// Non-finite input/output check (LP_ENONFINITE): one pass over a device
// array that records whether any element is an IEEE infinity or NaN.  The
// forward and adjoint recursions propagate a non-finite value to every later
// sample of the signal, and an unstable frozen filter overflows FP32 to inf
// (the conditioning point of the headline generator), so callers check
// their inputs before a call and their outputs after one.
#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

#include "tvlp.h"

namespace tvlp {
namespace {

constexpr int kCheckSlots = 64;      // concurrent checks (one result word each)
constexpr int kCheckThreads = 256;
__device__ unsigned g_nonfinite[kCheckSlots];
std::atomic<unsigned> g_next_slot{0};

// exponent field all ones: infinity or NaN (IEEE 754 binary32 / binary64)
__device__ __forceinline__ bool bad(float v) { return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u; }
__device__ __forceinline__ bool bad(double v) {
    return (static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7ff0000000000000ull) ==
           0x7ff0000000000000ull;
}

template <typename S>
__global__ void __launch_bounds__(kCheckThreads) k_nonfinite(const S *__restrict__ x, int64_t n, int64_t head,
                                                             unsigned *__restrict__ out) {
    // elements [0, head) and the tail past the last full 16-byte vector one
    // by one; the middle as 16-byte vectors
    constexpr int V = 16 / (int)sizeof(S);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool any = false;
    if (tid < head) any = bad(x[tid]);
    const int64_t nv = (n - head) / V;
    const S *xv = x + head;
    for (int64_t i = tid; i < nv; i += stride) {
        if constexpr (sizeof(S) == 4) {
            const float4 v = reinterpret_cast<const float4 *>(xv)[i];
            any |= bad(v.x) | bad(v.y) | bad(v.z) | bad(v.w);
        } else {
            const double2 v = reinterpret_cast<const double2 *>(xv)[i];
            any |= bad(v.x) | bad(v.y);
        }
    }
    const int64_t t0 = head + nv * V;
    if (t0 + tid < n) any |= bad(x[t0 + tid]);
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(out, 1u);
}

template <typename S>
int check_finite(const S *x, size_t n, void *stream) {
    if (n == 0) return LP_OK;
    if (x == nullptr) return LP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(x) % sizeof(S)) != 0) return LP_EALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *slots = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void **>(&slots), g_nonfinite) != cudaSuccess) return LP_ECUDA;
    unsigned *slot = slots + (g_next_slot.fetch_add(1) % kCheckSlots);
    if (cudaMemsetAsync(slot, 0, sizeof(unsigned), st) != cudaSuccess) return LP_ECUDA;
    // elements before the first 16-byte boundary (fewer than one vector)
    constexpr int V = 16 / (int)sizeof(S);
    const uintptr_t mis = reinterpret_cast<uintptr_t>(x) % 16;
    int64_t head = mis == 0 ? 0 : (int64_t)((16 - mis) / sizeof(S));
    if (head > (int64_t)n) head = (int64_t)n;
    const int64_t work = ((int64_t)n - head) / V + V + head;  // vectors plus single elements
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LP_ECUDA;
    int64_t blocks = (work + kCheckThreads - 1) / kCheckThreads;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_nonfinite<S><<<(unsigned)blocks, kCheckThreads, 0, st>>>(x, (int64_t)n, head, slot);
    if (cudaGetLastError() != cudaSuccess) return LP_ECUDA;
    unsigned found = 0;
    if (cudaMemcpyAsync(&found, slot, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LP_ECUDA;
    return found != 0 ? LP_ENONFINITE : LP_OK;
}

}  // namespace
}  // namespace tvlp

extern "C" int lp_tv_check_finite_f32(const float *x, size_t n, void *stream) {
    return tvlp::check_finite<float>(x, n, stream);
}

extern "C" int lp_tv_check_finite_f64(const double *x, size_t n, void *stream) {
    return tvlp::check_finite<double>(x, n, stream);
}
