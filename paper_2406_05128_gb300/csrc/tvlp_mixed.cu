// Mixed orders in one call: signals of different lengths and different
// orders M (Eq. 5 with each signal's own order) filtered by one launch per
// kernel role.
//
// The kernels are compiled per padded order MP (orders pad to 2, 4, 8, 12,
// 16, 22, 30, 32 with zero coefficients).  A mixed batch is split into
// classes of signals that share a padded order; every launch of the call
// covers all classes: its blocks are partitioned among the classes, and each
// block runs the body of its class's order (k1_body, rec_body, scan_body)
// on that class's signals, chunk tables and workspace.  Within a class a
// signal keeps its own real order (read per chunk from the order table), so
// an order-17 and an order-22 signal share the order-22 code.  A signal's
// results do not depend on the rest of the batch: its chunks and scan groups
// depend only on its own length and its class's chunk length.
//
// Layouts (caller-owned device memory):
//   offsets [n+1]  first row of every signal in the packed e, s, gs, ge
//   orders  [n]    M of every signal, 1..32
//   a, ga          signal b's coefficient rows (len_b rows of orders[b]
//                  values) start at element aoff[b] = sum over b' < b of
//                  len_b' * orders[b'] rounded up to a multiple of 4 (16
//                  bytes); lp_tv_mixed_coeff_offsets computes them
//   zi, gzi [n][32] initial state of signal b at zi[b*32 + j-1], j <= orders[b]
#include <stdint.h>
#include <string.h>

#include <atomic>

#include <cuda_runtime.h>

#include "tvlp.h"
#include "tvlp_impl.cuh"
#include "tvlp_mixed.h"

namespace tvlp {
namespace {

constexpr int kClassOrders[kMaxClasses] = {2, 4, 8, 12, 16, 22, 30, 32};
constexpr int kMixTableThreads = 1024;

int class_of_order(int M) {
    for (int k = 0; k < kMaxClasses; ++k)
        if (M <= kClassOrders[k]) return k;
    return -1;
}

// the padded order the kernels run a signal of order M at
__device__ __forceinline__ int padded_order_dev(int M) {
    return M <= 2 ? 2 : M <= 4 ? 4 : M <= 8 ? 8 : M <= 12 ? 12 : M <= 16 ? 16 : M <= 22 ? 22 : M <= 30 ? 30 : 32;
}


// ---------------------------------------------------------------------------
// Tables: block k < nc lists class k's signals (batch order kept) and the
// prefix sums of their chunks and scan groups; block nc computes the
// coefficient offsets aoff of every signal.
// ---------------------------------------------------------------------------
__device__ inline void block_scan3(long long (&v)[3], long long (&tot)[3]) {
    __shared__ long long sh[3][kMixTableThreads];
    const int t = threadIdx.x;
    for (int j = 0; j < 3; ++j) sh[j][t] = v[j];
    __syncthreads();
    for (int d = 1; d < kMixTableThreads; d <<= 1) {
        long long x[3];
        for (int j = 0; j < 3; ++j) x[j] = t >= d ? sh[j][t - d] : 0;
        __syncthreads();
        for (int j = 0; j < 3; ++j) sh[j][t] += x[j];
        __syncthreads();
    }
    for (int j = 0; j < 3; ++j) {
        tot[j] = sh[j][kMixTableThreads - 1];
        v[j] = sh[j][t] - v[j];  // exclusive
    }
    __syncthreads();
}

constexpr int kMixGradRows = 256;  // rows of one coefficient-gradient tile

__global__ void __launch_bounds__(kMixTableThreads)
    k_mixed_tables(MixLaunch ml, const int64_t *__restrict__ off, const int *__restrict__ ord, int n,
                   int64_t *__restrict__ aoff, int *__restrict__ tstart) {
    const int k = blockIdx.x, t = threadIdx.x;
    long long carry[3] = {0, 0, 0};
    if (k == ml.nc) {
        // coefficient offsets, and the first gradient tile of every signal
        for (int t0 = 0; t0 < n; t0 += kMixTableThreads) {
            const int g = t0 + t;
            long long v[3] = {0, 0, 0}, tot[3];
            if (g < n) {
                const int64_t len = off[g + 1] - off[g];
                v[0] = (len * (long long)ord[g] + 3) / 4 * 4;
                v[1] = (len + kMixGradRows - 1) / kMixGradRows;
            }
            block_scan3(v, tot);
            if (g < n) {
                aoff[g] = carry[0] + v[0];
                tstart[g] = (int)(carry[1] + v[1]);
            }
            carry[0] += tot[0];
            carry[1] += tot[1];
        }
        if (t == 0) {
            aoff[n] = carry[0];
            tstart[n] = (int)carry[1];
        }
        return;
    }
    const MixClass &c = ml.c[k];
    int *sig = const_cast<int *>(c.bt.sig);
    int *cstart = const_cast<int *>(c.bt.cstart);
    int *gstart = const_cast<int *>(c.bt.gstart);
    for (int t0 = 0; t0 < n; t0 += kMixTableThreads) {
        const int g = t0 + t;
        long long v[3] = {0, 0, 0}, tot[3];
        if (g < n && padded_order_dev(ord[g]) == c.MP) {
            const int64_t len = off[g + 1] - off[g];
            const int64_t ch = len > 0 ? (len + c.L - 1) / c.L : 0;
            v[0] = 1;
            v[1] = ch;
            v[2] = ch > 0 ? (ch + group_size(ch) - 1) / group_size(ch) : 0;
        }
        const bool member = v[0] != 0;
        block_scan3(v, tot);
        if (member) {
            const long long i = carry[0] + v[0];
            sig[i] = g;
            cstart[i] = (int)(carry[1] + v[1]);
            gstart[i] = (int)(carry[2] + v[2]);
        }
        for (int j = 0; j < 3; ++j) carry[j] += tot[j];
    }
    if (t == 0) {
        cstart[c.bt.n] = (int)carry[1];
        gstart[c.bt.n] = (int)carry[2];
    }
}

// Eq. 12 over one tile of kMixGradRows rows of one signal:
// ga_i(t) = -ge(t) s(t - i), i <= M of the signal, s(t - i) = zi[g][i-t-1]
// before the signal's start.  The tile's rows are built in shared memory
// (one row per thread) and leave as one contiguous run of rows*M values.
__global__ void __launch_bounds__(kMixGradRows)
    k_grad_a_mixed(const int64_t *__restrict__ off, const int *__restrict__ ord, const int64_t *__restrict__ aoff,
                   const int *__restrict__ tstart, int n, const float *__restrict__ ge, const float *__restrict__ s,
                   const float *__restrict__ zi, float *__restrict__ ga) {
    __shared__ float s_t[kMixGradRows + 32];
    __shared__ __align__(128) float tile[kMixGradRows * 32];
    const int g = find_signal(tstart, n, blockIdx.x);
    const int64_t o = __ldg(off + g), len = __ldg(off + g + 1) - o;
    const int64_t t0 = (int64_t)(blockIdx.x - __ldg(tstart + g)) * kMixGradRows;
    const int rows = (int)(len - t0 < kMixGradRows ? len - t0 : kMixGradRows);
    const int m = __ldg(ord + g);
    // s_t[i] = s(t0 - 32 + i) of the signal (zi before its start)
    for (int i = threadIdx.x; i < kMixGradRows + 32; i += blockDim.x) {
        const int64_t t = t0 - 32 + i;
        float v = 0.f;
        if (t >= 0 && t < len) v = s[o + t];
        else if (t < 0 && zi != nullptr && -t <= 32) v = zi[(int64_t)g * kMixLdz + (-t - 1)];
        s_t[i] = v;
    }
    __shared__ float g_t[kMixGradRows];
    pdl_wait();  // ge comes from the kernel just before
    pdl_release();
    const int r = threadIdx.x;
    g_t[r] = r < rows ? ge[o + t0 + r] : 0.f;
    __syncthreads();
    // element idx of the tile is row idx / m, coefficient idx % m + 1: a
    // thread per element keeps the shared stores conflict-free
    {
        // (row, coefficient) of the thread's element, advanced without a
        // division per element
        const int step_r = kMixGradRows / m, step_i = kMixGradRows - step_r * m;
        int rr = threadIdx.x / m, i = threadIdx.x - rr * m;
        for (int idx = threadIdx.x; idx < rows * m; idx += kMixGradRows) {
            tile[idx] = -g_t[rr] * s_t[32 + rr - i - 1];
            rr += step_r;
            i += step_i;
            if (i >= m) {
                i -= m;
                ++rr;
            }
        }
    }
    fence_proxy_async();
    __syncthreads();
    float *dst = ga + __ldg(aoff + g) + t0 * m;
    const unsigned bytes = (unsigned)(rows * m * sizeof(float));
    if (aligned16(dst) && bytes % 16 == 0) {
        // one bulk copy of the tile's rows
        if (threadIdx.x == 0) {
            bulk_store(dst, tile, bytes);
            bulk_store_commit_wait();
        }
    } else {
        for (int idx = threadIdx.x; idx < rows * m; idx += blockDim.x) dst[idx] = tile[idx];
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int MP> struct MixGeo {
    static constexpr size_t K1_SMEM = 8 * SumGeo<float, MP, Pack<MP>::G, Pack<MP>::R>::WARP_BYTES;
    static constexpr int K1_PER_BLOCK = 8 * SumGeo<float, MP, Pack<MP>::G, Pack<MP>::R>::CPW;
    static constexpr size_t REC_SMEM = RecGeo<float, MP, MixRecChunks<MP>::N>::SMEM;
    static constexpr int REC_CHUNKS = MixRecChunks<MP>::N;
    static constexpr size_t SCAN_SMEM = (size_t)kScanWarps * ScanGeo<float, MP, MixScanDepth<MP>::N>::WARP_BYTES;
};
struct ClassGeo {
    size_t k1_smem, rec_smem, scan_smem;
    int k1_per_block, rec_chunks;
};
ClassGeo class_geo(int MP) {
    switch (MP) {
#define TVLP_GEO(MPV) \
    case MPV:         \
        return {MixGeo<MPV>::K1_SMEM, MixGeo<MPV>::REC_SMEM, MixGeo<MPV>::SCAN_SMEM, MixGeo<MPV>::K1_PER_BLOCK, \
                MixGeo<MPV>::REC_CHUNKS};
        TVLP_GEO(2) TVLP_GEO(4) TVLP_GEO(8) TVLP_GEO(12) TVLP_GEO(16) TVLP_GEO(22) TVLP_GEO(30) TVLP_GEO(32)
#undef TVLP_GEO
    }
    return {0, 0, 0, 0, 1};
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Chunk length of a class when the caller passes 0: the single-order
// varlen call's pick for the class's signal count and mean length.
int class_chunk(int n_k, int64_t total_k, int MP) {
    const int c = lp_tv_pick_chunk(n_k, n_k > 0 ? cdiv(total_k, n_k) : 1, MP, LP_DTYPE_F32);
    return (int)(cdiv(c > 0 ? c : 16, 16) * 16);
}

// The host's view of a mixed call: classes, their problems and workspace.
struct MixPlan {
    int nc = 0;
    int n = 0;
    int64_t total = 0;
    int MPk[kMaxClasses];
    int cls_of_k[kMaxClasses];  // kClassOrders index of class k
    Problem p[kMaxClasses];
    int exact[kMaxClasses];
    size_t ws_class[kMaxClasses];
    int64_t tiles;  // coefficient-gradient tiles of the batch
    size_t off_aoff, off_tstart, off_sig, off_class[kMaxClasses], bytes;
};

int plan_mixed(int n, const int64_t *offsets_host, const int *orders_host, int chunk, MixPlan *mp) {
    if (n < 0 || chunk < 0) return LP_EINVAL;
    if (n > 0 && (offsets_host == nullptr || orders_host == nullptr)) return LP_EINVAL;
    MixPlan &P = *mp;
    P = MixPlan();
    P.n = n;
    int cnt[kMaxClasses] = {}, all_exact[kMaxClasses];
    int64_t rows[kMaxClasses] = {};
    for (int k = 0; k < kMaxClasses; ++k) all_exact[k] = 1;
    if (n > 0 && offsets_host[0] != 0) return LP_EINVAL;
    for (int b = 0; b < n; ++b) {
        const int M = orders_host[b];
        if (M < 1) return LP_EINVAL;
        const int k = class_of_order(M);
        if (k < 0) return LP_EUNSUPPORTED;
        const int64_t len = offsets_host[b + 1] - offsets_host[b];
        if (len < 0) return LP_EINVAL;
        ++cnt[k];
        rows[k] += len;
        if (M != kClassOrders[k]) all_exact[k] = 0;
    }
    P.total = n > 0 ? offsets_host[n] : 0;
    if (P.total >= (int64_t)INT32_MAX / 2) return LP_EUNSUPPORTED;
    for (int k = 0; k < kMaxClasses; ++k) {
        if (cnt[k] == 0) continue;
        const int c = P.nc++;
        P.cls_of_k[c] = k;
        P.MPk[c] = kClassOrders[k];
        P.exact[c] = all_exact[k];
        Problem &p = P.p[c];
        memset(&p, 0, sizeof(p));
        p.B = cnt[k];
        p.T = rows[k];
        p.M = kClassOrders[k];
        p.MP = kClassOrders[k];
        p.L = chunk > 0 ? (int)(cdiv(chunk, 16) * 16) : class_chunk(cnt[k], rows[k], p.MP);
        p.NQ = cdiv(rows[k], p.L) + cnt[k];
        p.items = p.NQ;
        p.off = reinterpret_cast<const int64_t *>(1);  // varlen layout (tables in region 8)
        P.ws_class[c] = ws_bytes(p, sizeof(float));
    }
    P.tiles = 0;
    for (int b = 0; b < n; ++b) P.tiles += cdiv(offsets_host[b + 1] - offsets_host[b], 256);
    size_t off = 0;
    P.off_aoff = off;
    off += align256((size_t)(n + 1) * sizeof(int64_t));
    P.off_tstart = off;
    off += align256((size_t)(n + 1) * sizeof(int));
    P.off_sig = off;
    off += align256((size_t)(n > 0 ? n : 1) * sizeof(int));
    for (int c = 0; c < P.nc; ++c) {
        P.off_class[c] = off;
        off += align256(P.ws_class[c]);
    }
    P.bytes = off;
    return LP_OK;
}

// Fill the launch descriptor for the call's device pointers.  The class
// signal lists share one array of n entries, class after class.
void fill_launch(const MixPlan &P, const int64_t *off, const int *ord, void *ws, MixLaunch *ml) {
    char *base = static_cast<char *>(ws);
    const int64_t *aoff = reinterpret_cast<const int64_t *>(base + P.off_aoff);
    int *sig = reinterpret_cast<int *>(base + P.off_sig);
    ml->nc = P.nc;
    int sig_at = 0;
    for (int c = 0; c < P.nc; ++c) {
        Problem p = P.p[c];
        p.off = off;
        void *cws = base + P.off_class[c];
        MixClass &m = ml->c[c];
        m.MP = p.MP;
        m.L = p.L;
        m.exact = P.exact[c];
        m.bt = batch_of(p, cws, sizeof(float));
        m.bt.sig = sig + sig_at;
        m.bt.ord = ord;
        m.bt.aoff = aoff;
        m.bt.ldz = kMixLdz;
        sig_at += p.B;
        m.NQ = p.NQ;
        m.items = p.items;
        m.Y = reinterpret_cast<float *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 0));
        m.X = reinterpret_cast<float *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 1));
        m.Z = reinterpret_cast<float *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 2));
        m.W = reinterpret_cast<float *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 3));
        m.GY = reinterpret_cast<float *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 4));
        m.GZ = reinterpret_cast<float *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 5));
        m.GX = reinterpret_cast<float *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 6));
        m.cnt = reinterpret_cast<unsigned *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 7));
        m.list = reinterpret_cast<int *>(static_cast<char *>(cws) + ws_offset(p, sizeof(float), 9));
    }
}

// block ranges of the classes for a launch with `per_class(c)` blocks each
template <typename F> int64_t assign_blocks(MixLaunch *ml, F per_class) {
    int64_t b0 = 0;
    for (int c = 0; c < ml->nc; ++c) {
        const int64_t nb = per_class(c);
        ml->c[c].block0 = b0;
        ml->c[c].nblocks = nb;
        b0 += nb;
    }
    return b0;
}

template <typename K> cudaError_t set_smem(K kern, size_t bytes, std::atomic<size_t> *done) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_acquire) >= bytes) return cudaSuccess;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err == cudaSuccess) done[dev].store(bytes, std::memory_order_release);
    return err;
}

MixRecKernel mix_rec_kernel(int mode) {
    MixRecKernel k = mix_rec_kernel_part0(mode);
    return k != nullptr ? k : mix_rec_kernel_part1(mode);
}
MixScanKernel mix_scan_kernel(int mode) {
    MixScanKernel k = mix_scan_kernel_part0(mode);
    return k != nullptr ? k : mix_scan_kernel_part1(mode);
}

cudaError_t mix_launch_k1(bool bwd, const MixLaunch &ml, unsigned grid, size_t smem, const float *a, const float *u,
                          int *status, cudaStream_t st) {
    static std::atomic<size_t> done[2][kMaxDevices] = {};
    MixK1Kernel kern = mix_k1_kernel(bwd);
    cudaError_t err = set_smem(kern, smem, done[bwd ? 1 : 0]);
    if (err != cudaSuccess) return err;
    return launch(kern, dim3(grid), dim3(256), smem, st, false, ml, a, u, 0, status);
}

cudaError_t mix_launch_rec(int mode, const MixLaunch &ml, unsigned grid, size_t smem, const float *a, const float *u,
                           const float *zi, float *out, float *gzi, int zero_cnt, int fix, int *status,
                           cudaStream_t st) {
    static std::atomic<size_t> done[4][kMaxDevices] = {};
    MixRecKernel kern = mix_rec_kernel(mode);
    if (kern == nullptr || mode < 0 || mode > 3) return cudaErrorInvalidValue;
    cudaError_t err = set_smem(kern, smem, done[mode]);
    if (err != cudaSuccess) return err;
    return launch(kern, dim3(grid), dim3(32), smem, st, false, ml, a, u, zi, out, gzi, zero_cnt, fix, 0, status);
}

cudaError_t mix_scan_occupancy(int mode, size_t smem, int *per_sm) {
    static std::atomic<size_t> done[6][kMaxDevices] = {};
    MixScanKernel kern = mix_scan_kernel(mode);
    if (kern == nullptr || mode < 0 || mode > 5) return cudaErrorInvalidValue;
    cudaError_t err = set_smem(kern, smem, done[mode]);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, kScanWarps * 32, smem);
}

cudaError_t mix_launch_scan(int mode, const MixLaunch &ml, unsigned grid, size_t smem, const float *zi, int *status,
                            cudaStream_t st) {
    MixScanKernel kern = mix_scan_kernel(mode);
    if (kern == nullptr) return cudaErrorInvalidValue;
    return launch(kern, dim3(grid), dim3(kScanWarps * 32), smem, st, true, ml, zi, status);
}

struct MixRun {
    const MixPlan &P;
    const MixLaunch &base;
    int *status;
    cudaStream_t st;

    cudaError_t tables(const int64_t *off, const int *ord, void *ws) const {
        char *b = static_cast<char *>(ws);
        k_mixed_tables<<<P.nc + 1, kMixTableThreads, 0, st>>>(base, off, ord, P.n,
                                                               reinterpret_cast<int64_t *>(b + P.off_aoff),
                                                               reinterpret_cast<int *>(b + P.off_tstart));
        return cudaGetLastError();
    }

    template <bool BWD> cudaError_t k1(const float *a, const float *u) const {
        MixLaunch ml = base;
        size_t smem = 0;
        const int64_t grid = assign_blocks(&ml, [&](int c) {
            const ClassGeo g = class_geo(ml.c[c].MP);
            smem = g.k1_smem > smem ? g.k1_smem : smem;
            return cdiv(ml.c[c].NQ, g.k1_per_block);
        });
        return mix_launch_k1(BWD, ml, (unsigned)grid, smem, a, u, status, st);
    }

    template <int MODE> cudaError_t rec(const float *a, const float *u, const float *zi, float *out, float *gzi,
                                        int zero_cnt, int fix) const {
        MixLaunch ml = base;
        size_t smem = 0;
        const int64_t grid = assign_blocks(&ml, [&](int c) {
            const ClassGeo g = class_geo(ml.c[c].MP);
            smem = g.rec_smem > smem ? g.rec_smem : smem;
            return cdiv(ml.c[c].NQ, g.rec_chunks);
        });
        return mix_launch_rec(MODE, ml, (unsigned)grid, smem, a, u, zi, out, gzi, zero_cnt, fix, status, st);
    }

    // cooperative: every block resident; the classes share the resident
    // blocks in proportion to their scan items (at least one block each)
    template <int MODE> cudaError_t scan(const float *zi) const {
        MixLaunch ml = base;
        size_t smem = 0;
        int64_t items = 0;
        for (int c = 0; c < ml.nc; ++c) {
            const ClassGeo g = class_geo(ml.c[c].MP);
            smem = g.scan_smem > smem ? g.scan_smem : smem;
            items += ml.c[c].items;
        }
        int dev = 0, per_sm = 0, sms = 0;
        cudaError_t err = cudaGetDevice(&dev);
        if (err != cudaSuccess) return err;
        if ((err = mix_scan_occupancy(MODE, smem, &per_sm)) != cudaSuccess) return err;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
        const int res = per_sm * sms;
        if (per_sm < 1 || res < ml.nc) return cudaErrorInvalidConfiguration;
        const int64_t grid = assign_blocks(&ml, [&](int c) {
            const int64_t want = cdiv(ml.c[c].items, kScanWarps);
            const int64_t share =
                items > 0 ? (int64_t)((double)(res - ml.nc) * (double)ml.c[c].items / (double)items) + 1 : 1;
            return share < want ? share : (want > 0 ? want : 1);
        });
        return mix_launch_scan(MODE, ml, (unsigned)grid, smem, zi, status, st);
    }
};

#define TVLP_MIX(K, CALL)                        \
    do {                                         \
        const int k_ = (K);                      \
        profile_mark(k_, false, st);             \
        if ((CALL) != cudaSuccess) return LP_ECUDA; \
        profile_mark(k_, true, st);              \
    } while (0)

int check_mixed_pointers(const void *p, size_t align) {
    return (reinterpret_cast<uintptr_t>(p) % align) == 0 ? LP_OK : LP_EALIGN;
}

}  // namespace
}  // namespace tvlp

using namespace tvlp;

extern "C" int64_t lp_tv_mixed_coeff_offsets(int n, const int64_t *offsets_host, const int *orders_host,
                                             int64_t *aoff_host) {
    if (n < 0 || (n > 0 && (offsets_host == nullptr || orders_host == nullptr))) return -1;
    int64_t acc = 0;
    for (int b = 0; b < n; ++b) {
        if (aoff_host != nullptr) aoff_host[b] = acc;
        const int64_t len = offsets_host[b + 1] - offsets_host[b];
        if (len < 0 || orders_host[b] < 0) return -1;
        acc += (len * orders_host[b] + 3) / 4 * 4;
    }
    if (aoff_host != nullptr) aoff_host[n] = acc;
    return acc;
}

extern "C" size_t lp_tv_workspace_bytes_mixed(int n, const int64_t *offsets_host, const int *orders_host,
                                              int chunk) {
    MixPlan P;
    if (plan_mixed(n, offsets_host, orders_host, chunk, &P) != LP_OK) return 0;
    return P.bytes;
}

extern "C" int lp_tv_forward_mixed_f32(int n, const int64_t *offsets, const int *orders,
                                       const int64_t *offsets_host, const int *orders_host, const float *a,
                                       const float *e, const float *zi, float *s, int chunk, void *workspace,
                                       size_t workspace_bytes, void *stream) {
    MixPlan P;
    int rc = plan_mixed(n, offsets_host, orders_host, chunk, &P);
    if (rc != LP_OK) return rc;
    if (n == 0 || P.total == 0) return LP_OK;
    if (offsets == nullptr || orders == nullptr || a == nullptr || e == nullptr || s == nullptr) return LP_EINVAL;
    if (check_mixed_pointers(offsets, 8) || check_mixed_pointers(orders, 4) || check_mixed_pointers(a, 16) ||
        check_mixed_pointers(e, 4) || check_mixed_pointers(s, 4) || check_mixed_pointers(zi, 4))
        return LP_EALIGN;
    if (workspace == nullptr || workspace_bytes < P.bytes || check_mixed_pointers(workspace, 256))
        return LP_EWORKSPACE;
    int *status = device_status_word();
    if (status == nullptr) return LP_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MixLaunch ml;
    fill_launch(P, offsets, orders, workspace, &ml);
    const MixRun run{P, ml, status, st};
    if (run.tables(offsets, orders, workspace) != cudaSuccess) return LP_ECUDA;
    TVLP_MIX(0, (run.k1<false>(a, e)));
    TVLP_MIX(1, (run.scan<CH_FWD>(zi)));
    TVLP_MIX(2, (run.rec<FWD_RERUN>(a, e, zi, s, nullptr, 0, 1)));
    TVLP_MIX(3, (run.scan<CH_FWD_FIX>(nullptr)));
    TVLP_MIX(4, (run.rec<FWD_RERUN>(a, e, zi, s, nullptr, 0, 2)));
    return LP_OK;
}

extern "C" int lp_tv_backward_mixed_f32(int n, const int64_t *offsets, const int *orders,
                                        const int64_t *offsets_host, const int *orders_host, const float *gs,
                                        const float *a, const float *s, const float *zi, float *ge, float *ga,
                                        float *gzi, int chunk, int flags, void *workspace, size_t workspace_bytes,
                                        void *stream) {
    if ((flags & ~LP_BWD_REUSE_FORWARD) != 0) return LP_EINVAL;
    MixPlan P;
    int rc = plan_mixed(n, offsets_host, orders_host, chunk, &P);
    if (rc != LP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n > 0 && P.total == 0) {
        if (gzi != nullptr && cudaMemsetAsync(gzi, 0, (size_t)n * kMixLdz * sizeof(float), st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if (n == 0) return LP_OK;
    if (offsets == nullptr || orders == nullptr || a == nullptr || gs == nullptr || ge == nullptr ||
        (ga != nullptr && s == nullptr))
        return LP_EINVAL;
    if (check_mixed_pointers(offsets, 8) || check_mixed_pointers(orders, 4) || check_mixed_pointers(a, 16) ||
        check_mixed_pointers(gs, 4) || check_mixed_pointers(ge, 4) || check_mixed_pointers(s, 4) ||
        check_mixed_pointers(zi, 4) || check_mixed_pointers(ga, 4) || check_mixed_pointers(gzi, 4))
        return LP_EALIGN;
    if (workspace == nullptr || workspace_bytes < P.bytes || check_mixed_pointers(workspace, 256))
        return LP_EWORKSPACE;
    int *status = device_status_word();
    if (status == nullptr) return LP_ECUDA;
    MixLaunch ml;
    fill_launch(P, offsets, orders, workspace, &ml);
    const MixRun run{P, ml, status, st};
    if (run.tables(offsets, orders, workspace) != cudaSuccess) return LP_ECUDA;
    int k = 0;
    if (flags & LP_BWD_REUSE_FORWARD) {
        // the forward's maps are in the workspace: one zero-state recursion
        // per chunk, then the transposed scan
        TVLP_MIX(k++, (run.rec<BWD_ZERO>(a, gs, nullptr, nullptr, nullptr, 1, 0)));
        TVLP_MIX(k++, (run.scan<CH_TRANS>(nullptr)));
    } else {
        TVLP_MIX(k++, (run.k1<true>(a, gs)));
        TVLP_MIX(k++, (run.scan<CH_BWD>(nullptr)));
    }
    TVLP_MIX(k++, (run.rec<BWD_RERUN>(a, gs, zi, ge, gzi, 0, 1)));
    if (flags & LP_BWD_REUSE_FORWARD)
        TVLP_MIX(k++, (run.scan<CH_TRANS_FIX>(nullptr)));
    else
        TVLP_MIX(k++, (run.scan<CH_BWD_FIX>(nullptr)));
    TVLP_MIX(k++, (run.rec<BWD_RERUN>(a, gs, zi, ge, gzi, 0, 2)));
    if (ga != nullptr) {
        char *b = static_cast<char *>(workspace);
        const int64_t *aoff = reinterpret_cast<const int64_t *>(b + P.off_aoff);
        const int *tstart = reinterpret_cast<const int *>(b + P.off_tstart);
        TVLP_MIX(k, (launch(k_grad_a_mixed, dim3((unsigned)P.tiles), dim3(kMixGradRows), 0, st, false, offsets, orders,
                            aoff, tstart, n, ge, s, zi, ga)));
    }
    return LP_OK;
}
#undef TVLP_MIX
