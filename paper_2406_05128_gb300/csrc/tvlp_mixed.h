// Shared declarations of the mixed-order calls (tvlp_mixed*.cu): the launch
// descriptor of a fused launch over the classes of a batch, and the host
// launchers of the fused kernels, each in a translation unit of its own so
// the build compiles them in parallel.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

#include "tvlp_impl.h"
#include "tvlp_kernels.cuh"

namespace tvlp {

constexpr int kMaxClasses = 8;
constexpr int kMixLdz = 32;  // initial-state stride per signal

// Chunks per warp of the mixed re-run passes: the orders above 22 take
// fewer, so every order's block needs about the shared memory of order 22's
// (a launch gives all its blocks the largest order's share, and fewer
// resident blocks would starve the bandwidth-bound passes).
template <int MP> struct MixRecChunks {
    static constexpr int N = MP > 22 ? 11 : kRecChunks;
};
// Map slots per warp of the mixed scans, for the same reason: the maps of
// the orders above 22 take twice the space, so they stream in batches of 2.
template <int MP> struct MixScanDepth {
    static constexpr int N = MP > 22 ? 4 : kScanDepth;
};

// One class of a mixed launch: its padded order, chunk length, batch view
// (class-local tables, the batch's offsets and orders), workspace regions,
// and the range of the launch's blocks that run it.
struct MixClass {
    int MP, L, exact;
    Batch bt;
    int64_t NQ, items;
    int64_t block0, nblocks;
    float *Y, *X, *Z, *W, *GY, *GZ, *GX;
    unsigned *cnt;
    int *list;
};
struct MixLaunch {
    int nc;
    MixClass c[kMaxClasses];
};


// the class of block `blk` of a fused launch
__device__ __forceinline__ int mix_class(const MixLaunch &ml, int64_t blk) {
    int k = 0;
    while (k + 1 < ml.nc && blk >= ml.c[k + 1].block0) ++k;
    return k;
}

// The fused kernels, each defined in a translation unit of its own (or a
// part of one, so the build compiles them in parallel); nullptr for a mode
// that part does not hold.
using MixK1Kernel = void (*)(MixLaunch, const float *, const float *, int, int *);
// fix: 0 none, 1 pass 1 (defects, scale), 2 pass 2 (listed chunks)
using MixRecKernel = void (*)(MixLaunch, const float *, const float *, const float *, float *, float *, int, int, int,
                              int *);
using MixScanKernel = void (*)(MixLaunch, const float *, int *);
MixK1Kernel mix_k1_kernel(bool bwd);
MixRecKernel mix_rec_kernel_part0(int mode);  // FWD_RERUN
MixRecKernel mix_rec_kernel_part1(int mode);  // BWD_ZERO, BWD_RERUN
MixScanKernel mix_scan_kernel_part0(int mode);  // CH_FWD, CH_BWD, CH_TRANS
MixScanKernel mix_scan_kernel_part1(int mode);  // the correction scans

}  // namespace tvlp
