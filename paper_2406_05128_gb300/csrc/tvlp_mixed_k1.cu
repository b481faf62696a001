// Fused mixed-order launch of the chunk summaries (see tvlp_mixed.cu).
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

template <bool BWD>
__global__ void __launch_bounds__(256, 1)
    k1_mixed(MixLaunch ml, const float *__restrict__ a, const float *__restrict__ u, int l2, int *__restrict__ status) {
    const int k = mix_class(ml, blockIdx.x);
    const MixClass &c = ml.c[k];
    const int64_t bid = (int64_t)blockIdx.x - c.block0;
#define TVLP_K1_CASE(MPV)                                                                                      \
    case MPV:                                                                                                  \
        k1_body<float, MPV, Pack<MPV>::G, Pack<MPV>::R, BWD, SRC_STREAM>(bid, c.bt, MPV, c.L, c.NQ, a, u, c.Y, \
                                                                         c.exact, c.cnt, c.bt.n + 1, l2,      \
                                                                         status, CoefSrc());                   \
        break;
    TVLP_MIX_SWITCH(TVLP_K1_CASE)
#undef TVLP_K1_CASE
}

#undef TVLP_MIX_SWITCH

}  // namespace

MixK1Kernel mix_k1_kernel(bool bwd) { return bwd ? k1_mixed<true> : k1_mixed<false>; }
}  // namespace tvlp
