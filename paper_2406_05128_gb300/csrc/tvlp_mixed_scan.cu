// Fused mixed-order launch of the two-level scans (see tvlp_mixed.cu).
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

template <int MODE>
__global__ void __launch_bounds__(kScanWarps * 32)
    k2_scan_mixed(MixLaunch ml, const float *__restrict__ zi, int *__restrict__ status) {
    const int k = mix_class(ml, blockIdx.x);
    const MixClass &c = ml.c[k];
    const int64_t bid = (int64_t)blockIdx.x - c.block0;
    constexpr bool FIX = ScanMode<MODE>::FIX;
    constexpr bool BWD = ScanMode<MODE>::REV;
    // main scans: maps Y (and the adjoint's zero-state summaries Z), states
    // out to X (forward) or W (adjoint); correction scans: defects in Z,
    // corrections to the region the direction's re-run does not read
    const float *Zin = (MODE == CH_FWD || MODE == CH_BWD) ? nullptr : c.Z;
    float *Xout = FIX ? (BWD ? c.X : c.W) : (BWD ? c.W : c.X);
#define TVLP_SCAN_CASE(MPV)                                                                                      \
    case MPV:                                                                                                    \
        scan_body<float, MPV, MODE, MixScanDepth<MPV>::N>(bid, c.nblocks, c.bt, MPV, c.items, c.Y, Zin, c.GY, c.GZ, c.GX,              \
                                    MODE == CH_FWD ? zi : nullptr, Xout, nullptr, c.cnt, status, c.list);        \
        break;
    TVLP_MIX_SWITCH(TVLP_SCAN_CASE)
#undef TVLP_SCAN_CASE
}
#undef TVLP_MIX_SWITCH

}  // namespace

// Compiled in two parts (TVLP_MIX_PART 0: the main scans; 1: the
// correction scans) so the build runs them in parallel.
#if TVLP_MIX_PART == 0
MixScanKernel mix_scan_kernel_part0(int mode) {
    switch (mode) {
        case CH_FWD: return k2_scan_mixed<CH_FWD>;
        case CH_BWD: return k2_scan_mixed<CH_BWD>;
        case CH_TRANS: return k2_scan_mixed<CH_TRANS>;
    }
    return nullptr;
}
#else
MixScanKernel mix_scan_kernel_part1(int mode) {
    switch (mode) {
        case CH_FWD_FIX: return k2_scan_mixed<CH_FWD_FIX>;
        case CH_TRANS_FIX: return k2_scan_mixed<CH_TRANS_FIX>;
        case CH_BWD_FIX: return k2_scan_mixed<CH_BWD_FIX>;
    }
    return nullptr;
}
#endif
}  // namespace tvlp
