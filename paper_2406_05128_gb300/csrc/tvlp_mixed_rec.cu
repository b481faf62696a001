// Fused mixed-order launch of the one-recursion passes (see tvlp_mixed.cu).
#include "tvlp_impl.cuh"
#include "tvlp_mixed.h"

namespace tvlp {
namespace {

#define TVLP_MIX_SWITCH(MPV_CASE) \
    switch (c.MP) {               \
        MPV_CASE(2)               \
        MPV_CASE(4)               \
        MPV_CASE(8)               \
        MPV_CASE(12)              \
        MPV_CASE(16)              \
        MPV_CASE(22)              \
        MPV_CASE(30)              \
        MPV_CASE(32)              \
        default: break;           \
    }

// fix: 0 none, 1 pass 1 (defects, scale), 2 pass 2 (listed chunks)
template <int MODE>
__global__ void __launch_bounds__(32)
    k_rec_mixed(MixLaunch ml, const float *__restrict__ a, const float *__restrict__ u, const float *__restrict__ zi,
                float *__restrict__ out, float *__restrict__ gzi, int zero_cnt, int fix, int l2,
                int *__restrict__ status) {
    const int k = mix_class(ml, blockIdx.x);
    const MixClass &c = ml.c[k];
    const int64_t bid = (int64_t)blockIdx.x - c.block0;
    constexpr bool BWD = MODE != FWD_RERUN;
    // incoming states: the forward's X, the adjoint's W; corrections in the
    // state region the direction does not use
    const float *Xin = MODE == BWD_ZERO ? nullptr : (BWD ? c.W : c.X);
    Fix<float> fx;
    if (fix == 1) {
        fx.D = c.Z;
        fx.scale = c.cnt;
    } else if (fix == 2) {
        fx.E = BWD ? c.X : c.W;
        fx.scale = c.cnt;
        fx.list = c.list;
        fx.list_n = c.cnt + (int64_t)c.bt.n * kCntStride;
    }
    float *Zout = MODE == BWD_ZERO ? c.Z : nullptr;
    unsigned *cnt = zero_cnt ? c.cnt : nullptr;
    const int reverse = (MODE == BWD_ZERO) ? 0 : 1;
#define TVLP_REC_CASE(MPV)                                                                                            \
    case MPV:                                                                                                         \
        if (c.exact)                                                                                                  \
            rec_body<float, MPV, true, MODE, SRC_STREAM, MixRecChunks<MPV>::N>(bid, c.nblocks, c.bt, MPV, c.L, c.NQ, a, u, Xin, zi, out,    \
                                                         Zout, gzi, reverse, cnt, c.bt.n + 1, l2, MPV, status,        \
                                                         CoefSrc(), nullptr, nullptr, fx);                            \
        else                                                                                                          \
            rec_body<float, MPV, false, MODE, SRC_STREAM, MixRecChunks<MPV>::N>(bid, c.nblocks, c.bt, MPV, c.L, c.NQ, a, u, Xin, zi, out,   \
                                                          Zout, gzi, reverse, cnt, c.bt.n + 1, l2, MPV, status,       \
                                                          CoefSrc(), nullptr, nullptr, fx);                           \
        break;
    TVLP_MIX_SWITCH(TVLP_REC_CASE)
#undef TVLP_REC_CASE
}

#undef TVLP_MIX_SWITCH

}  // namespace

// Compiled in two parts (TVLP_MIX_PART 0: the forward re-run; 1: the
// adjoint's passes) so the build runs them in parallel.
#if TVLP_MIX_PART == 0
MixRecKernel mix_rec_kernel_part0(int mode) { return mode == FWD_RERUN ? k_rec_mixed<FWD_RERUN> : nullptr; }
#else
MixRecKernel mix_rec_kernel_part1(int mode) {
    return mode == BWD_ZERO ? k_rec_mixed<BWD_ZERO> : mode == BWD_RERUN ? k_rec_mixed<BWD_RERUN> : nullptr;
}
#endif
}  // namespace tvlp
