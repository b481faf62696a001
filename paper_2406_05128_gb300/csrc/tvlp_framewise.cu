// Frame-wise overlap-add approximation of the time-varying LP filter: the
// method of the earlier GOLF work that the sample-wise filter of Eq. 5
// replaces (Sec. 3.2), kept here for the training-speed comparison of
// Sec. 4.3 (GOLF-ss against the frame-wise GOLF-ff; 75 % overlap, Sec. 5.2).
//
// Frames of N = 4*hop samples start every hop samples; frame f covers
// samples t_f .. t_f + N - 1, t_f = (f - 3)*hop, F = ceil(T/hop) + 3 frames.
//   forward   u_f(n) = w(n) e(t_f + n),  y_f = 1/A_f(z) u_f from zero state
//             (Eq. 2 with the frame's coefficients af[f]), s(t) = sum_f y_f(t - t_f)
//   adjoint   gu_f = Eq. 11 with af[f] over the frame on g_f(n) = gs(t_f + n),
//             ge(t) = sum_f w(t - t_f) gu_f(t - t_f),
//             gaf[f][i-1] = -sum_n gu_f(n) y_f(n - i)   (Eq. 12 summed, Eq. 3)
//   w(n) = (1 - cos(2 pi n / N)) / 4: the four windows over a sample sum to 1.
//
// GPU mapping.  One warp per group of 32 consecutive frames of one signal;
// lane t runs frame h0 + t (its recursion is sequential, 4 hops long).  The
// group owns the 29 output hops h0 .. h0+28, every frame of which it runs
// (the last three frames are also run by the next group), so the overlap-add
// happens in shared memory, in a fixed order, with no atomics: the input
// hops the frames read are staged once, and the frame outputs accumulate
// hop by hop, lane t adding to hop t + p in phase p (distinct hops per
// phase, a warp barrier between phases).  Hop rows are padded to an odd
// length so that the 32 lanes hit 32 banks.  The forward also keeps every
// frame output y[b][n][f] (frames fastest: each step's stores are one
// coalesced line per warp) for the adjoint's coefficient gradient.
#include <stdint.h>

#include <cuda_runtime.h>

#include "tvlp.h"
#include "tvlp_kernels.cuh"

namespace tvlp {
namespace {

constexpr int kFwFrames = 32;            // frames per warp (lanes)
constexpr int kFwOwned = kFwFrames - 3;  // output hops a warp owns
constexpr int kFwHops = kFwFrames + 3;   // input / output hops a warp touches
constexpr int kFwMaxHop = 512;

__host__ __device__ inline int fw_row(int hop) { return hop | 1; }  // odd row length (banks)

__host__ __device__ inline size_t fw_smem(int hop) {
    return (size_t)(2 * kFwHops * fw_row(hop) + 4 * hop) * sizeof(float);
}

// Stage hops [h0 - 3, h0 + 32) of x (one signal, T samples) into rows of `row`
// floats: rel[r][j] = x((h0 - 3 + r) hop + j), zero outside 0 .. T-1.
__device__ inline void fw_stage(float *rel, const float *__restrict__ x, int64_t T, int64_t h0, int hop, int row,
                               int lane) {
    for (int r = 0; r < kFwHops; ++r) {
        const int64_t t0 = (h0 - 3 + r) * (int64_t)hop;
        for (int j = lane; j < hop; j += 32) {
            const int64_t t = t0 + j;
            rel[r * row + j] = (t >= 0 && t < T) ? __ldg(x + t) : 0.f;
        }
    }
}

// the owned hops' rows of `acc` out to x (samples below T)
__device__ inline void fw_store(float *__restrict__ x, const float *acc, int64_t T, int64_t h0, int hop, int row,
                                int lane) {
    for (int r = 3; r < 3 + kFwOwned; ++r) {
        const int64_t t0 = (h0 - 3 + r) * (int64_t)hop;
        for (int j = lane; j < hop; j += 32) {
            const int64_t t = t0 + j;
            if (t < T) x[t] = acc[r * row + j];
        }
    }
}

__device__ inline void fw_window(float *win, int hop, int lane) {
    const int N = 4 * hop;
    for (int n = lane; n < N; n += 32) win[n] = 0.25f * (1.f - cospif(2.f * (float)n / (float)N));
}

template <int MP>
__device__ inline void fw_coeffs(float (&c)[MP], const float *__restrict__ af, int64_t F, int M, int64_t b, int64_t f,
                                 bool valid) {
#pragma unroll
    for (int i = 0; i < MP; ++i) c[i] = (valid && i < M) ? __ldg(af + (b * F + f) * M + i) : 0.f;
}

template <int MP>
__global__ void __launch_bounds__(32, 1) k_fw_forward(int64_t T, int M, int hop, int64_t F, const float *__restrict__ af,
                                                   const float *__restrict__ e, float *__restrict__ s,
                                                   float *__restrict__ y) {
    extern __shared__ __align__(16) float fw_sm[];
    const int lane = threadIdx.x, row = fw_row(hop), N = 4 * hop;
    const int64_t b = blockIdx.y, h0 = (int64_t)blockIdx.x * kFwOwned, f = h0 + lane;
    float *in = fw_sm, *acc = fw_sm + kFwHops * row, *win = acc + kFwHops * row;
    fw_window(win, hop, lane);
    fw_stage(in, e + b * T, T, h0, hop, row, lane);
    for (int i = lane; i < kFwHops * row; i += 32) acc[i] = 0.f;
    const bool valid = f < F;
    float c[MP];
    fw_coeffs<MP>(c, af, F, M, b, f, valid);
    __syncwarp();
    constexpr int WIN = MP + SR;
    float h[WIN];
#pragma unroll
    for (int m = 0; m < WIN; ++m) h[m] = 0.f;
    float *yb = y != nullptr ? y + b * (int64_t)N * F : nullptr;
    for (int p = 0; p < 4; ++p) {
        const float *ir = in + (lane + p) * row;
        float *orow = acc + (lane + p) * row;
#pragma unroll 1
        for (int j0 = 0; j0 < hop; j0 += SR) {
            // the block's inputs first, its outputs after: no shared-memory
            // access waits inside the recursion
            float uu[SR], vv[SR];
#pragma unroll
            for (int j = 0; j < SR; ++j) uu[j] = valid ? win[p * hop + j0 + j] * ir[j0 + j] : 0.f;
#pragma unroll
            for (int j = 0; j < SR; ++j) vv[j] = fwd_step_win<float, MP, WIN>(h, c, uu[j], j);
#pragma unroll
            for (int j = 0; j < SR; ++j) {
                orow[j0 + j] += vv[j];
                if (yb != nullptr && valid) yb[(int64_t)(p * hop + j0 + j) * F + f] = vv[j];
            }
            slide<float, MP, WIN>(h);
        }
        __syncwarp();  // hop lane + p + 1 is lane + 1's in this phase
    }
    fw_store(s + b * T, acc, T, h0, hop, row, lane);
}

template <int MP>
__global__ void __launch_bounds__(32, 1) k_fw_backward(int64_t T, int M, int hop, int64_t F, const float *__restrict__ af,
                                                    const float *__restrict__ y, const float *__restrict__ gs,
                                                    float *__restrict__ ge, float *__restrict__ gaf) {
    extern __shared__ __align__(16) float fw_sm[];
    const int lane = threadIdx.x, row = fw_row(hop), N = 4 * hop;
    const int64_t b = blockIdx.y, h0 = (int64_t)blockIdx.x * kFwOwned, f = h0 + lane;
    float *in = fw_sm, *acc = fw_sm + kFwHops * row, *win = acc + kFwHops * row;
    fw_window(win, hop, lane);
    fw_stage(in, gs + b * T, T, h0, hop, row, lane);
    for (int i = lane; i < kFwHops * row; i += 32) acc[i] = 0.f;
    const bool valid = f < F;
    float c[MP];
    fw_coeffs<MP>(c, af, F, M, b, f, valid);
    __syncwarp();
    constexpr int WIN = MP + SR;
    // adjoint window q (see bwd_step_win) and the forward outputs the
    // coefficient gradient pairs with each step: at the start of a block of
    // steps n = nh, nh-1, .., nh-SR+1, yw[k] = y_f(nh - 1 - k)
    float q[WIN], yw[WIN], g[MP];
#pragma unroll
    for (int m = 0; m < WIN; ++m) q[m] = 0.f;
#pragma unroll
    for (int i = 0; i < MP; ++i) g[i] = 0.f;
    const float *yb = y + b * (int64_t)N * F;
    auto y_at = [&](int n) -> float { return (valid && n >= 0) ? __ldg(yb + (int64_t)n * F + f) : 0.f; };
#pragma unroll
    for (int k = 0; k < WIN; ++k) yw[k] = y_at(N - 1 - 1 - k);
    for (int p = 3; p >= 0; --p) {
        const float *ir = in + (lane + p) * row;
        float *orow = acc + (lane + p) * row;
#pragma unroll 1
        for (int j0 = hop - SR; j0 >= 0; j0 -= SR) {
            const int nh = p * hop + j0 + SR - 1;  // first (latest) step of the block
            float uu[SR], vv[SR];
#pragma unroll
            for (int j = 0; j < SR; ++j) uu[j] = valid ? ir[j0 + SR - 1 - j] : 0.f;
#pragma unroll
            for (int j = 0; j < SR; ++j) {
                const float v = bwd_step_win<float, MP, WIN>(q, c, uu[j], j);
                vv[j] = v;
#pragma unroll
                for (int i = 1; i <= MP; ++i) g[i - 1] = fmaf(-v, yw[j + i - 1], g[i - 1]);
            }
#pragma unroll
            for (int j = 0; j < SR; ++j) orow[j0 + SR - 1 - j] += win[nh - j] * vv[j];
            slide<float, MP, WIN>(q);
#pragma unroll
            for (int k = 0; k < WIN - SR; ++k) yw[k] = yw[k + SR];
#pragma unroll
            for (int k = WIN - SR; k < WIN; ++k) yw[k] = y_at(nh - SR - 1 - k);
        }
        __syncwarp();
    }
    fw_store(ge + b * T, acc, T, h0, hop, row, lane);
    if (valid && lane < kFwOwned) {
        for (int i = 0; i < M; ++i) gaf[(b * F + f) * M + i] = g[i];
    }
}

int padded_order(int M) {
    static const int mp[] = {2, 4, 8, 12, 16, 22, 30, 32};
    for (int v : mp)
        if (M <= v) return v;
    return -1;
}

int fw_check(int B, int64_t T, int M, int hop) {
    if (B < 0 || T < 0 || M < 0) return LP_EINVAL;
    if (hop < SR || hop > kFwMaxHop || hop % SR != 0) return LP_EINVAL;
    if (M > 32) return LP_EUNSUPPORTED;
    if (T >= (int64_t)1 << 31) return LP_EUNSUPPORTED;
    return LP_OK;
}

template <int MP> cudaError_t fw_launch(bool fwd, int B, int64_t T, int M, int hop, const float *af, const float *e,
                                         float *s, float *y, const float *gs, float *ge, float *gaf,
                                         cudaStream_t st) {
    const int64_t F = (T + hop - 1) / hop + 3;
    const int64_t hops = (T + hop - 1) / hop;
    const dim3 grid((unsigned)((hops + kFwOwned - 1) / kFwOwned), (unsigned)B);
    const size_t smem = fw_smem(hop);
    if (fwd) {
        cudaError_t err = cudaFuncSetAttribute(k_fw_forward<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k_fw_forward<MP><<<grid, 32, smem, st>>>(T, M, hop, F, af, e, s, y);
    } else {
        cudaError_t err = cudaFuncSetAttribute(k_fw_backward<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k_fw_backward<MP><<<grid, 32, smem, st>>>(T, M, hop, F, af, y, gs, ge, gaf);
    }
    return cudaGetLastError();
}

int fw_dispatch(bool fwd, int B, int64_t T, int M, int hop, const float *af, const float *e, float *s, float *y,
                const float *gs, float *ge, float *gaf, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaErrorInvalidValue;
    switch (padded_order(M)) {
#define TVLP_FW(MPV)                                                               \
    case MPV:                                                                      \
        err = fw_launch<MPV>(fwd, B, T, M, hop, af, e, s, y, gs, ge, gaf, st);     \
        break;
        TVLP_FW(2) TVLP_FW(4) TVLP_FW(8) TVLP_FW(12) TVLP_FW(16) TVLP_FW(22) TVLP_FW(30) TVLP_FW(32)
#undef TVLP_FW
        default:
            return LP_EUNSUPPORTED;
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        return LP_ECUDA;
    }
    return LP_OK;
}

}  // namespace
}  // namespace tvlp

using namespace tvlp;

extern "C" int64_t lp_framewise_num_frames(int64_t T, int hop) {
    if (T < 0 || hop < 1) return -1;
    return (T + hop - 1) / hop + 3;
}

extern "C" size_t lp_framewise_outputs_bytes(int B, int64_t T, int hop) {
    if (B < 0 || T < 0 || hop < 1) return 0;
    return (size_t)B * 4 * (size_t)hop * (size_t)((T + hop - 1) / hop + 3) * sizeof(float);
}

extern "C" int lp_framewise_forward_f32(int B, int64_t T, int M, int hop, const float *af, const float *e, float *s,
                                        float *y, void *stream) {
    int rc = fw_check(B, T, M, hop);
    if (rc != LP_OK) return rc;
    if (B == 0 || T == 0) return LP_OK;
    if (e == nullptr || s == nullptr || (M > 0 && af == nullptr)) return LP_EINVAL;
    // M == 0 runs the smallest order with zero coefficients: s is the
    // overlap-add of the windowed frames, e up to rounding
    return fw_dispatch(true, B, T, M, hop, af, e, s, y, nullptr, nullptr, nullptr, stream);
}

extern "C" int lp_framewise_backward_f32(int B, int64_t T, int M, int hop, const float *af, const float *y,
                                         const float *gs, float *ge, float *gaf, void *stream) {
    int rc = fw_check(B, T, M, hop);
    if (rc != LP_OK) return rc;
    if (B == 0 || T == 0) return LP_OK;
    if (gs == nullptr || ge == nullptr || y == nullptr || (M > 0 && (af == nullptr || gaf == nullptr)))
        return LP_EINVAL;
    return fw_dispatch(false, B, T, M, hop, af, nullptr, nullptr, const_cast<float *>(y), gs, ge, gaf, stream);
}
