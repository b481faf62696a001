// C ABI of the time-varying LP library: argument checks, chunk selection
// and dispatch to the per-order instantiations (see include/tvlp.h).
#include <atomic>
#include <cmath>
#include <limits.h>
#include <stdint.h>
#include <string.h>

#include "tvlp.h"
#include "tvlp_impl.h"

namespace tvlp {
extern template struct Impl<float, 2>;
extern template struct Impl<float, 4>;
extern template struct Impl<float, 8>;
extern template struct Impl<float, 12>;
extern template struct Impl<float, 16>;
extern template struct Impl<float, 22>;
extern template struct Impl<float, 30>;
extern template struct Impl<float, 32>;
extern template struct Impl<double, 2>;
extern template struct Impl<double, 4>;
extern template struct Impl<double, 8>;
extern template struct Impl<double, 12>;
extern template struct Impl<double, 16>;
}  // namespace tvlp

// Device status word: kernels record a bounded wait that gave up here.
__device__ int g_tvlp_status = 0;

namespace tvlp {
namespace {
thread_local void **g_prof_events = nullptr;
thread_local int g_prof_n = 0;
thread_local LaunchShape g_shape = {1, 16};
}  // namespace

LaunchShape launch_shape() { return g_shape; }

void profile_mark(int k, bool end, cudaStream_t st) {
    if (g_prof_events == nullptr || k < 0 || k >= g_prof_n) return;
    cudaEvent_t ev = static_cast<cudaEvent_t>(g_prof_events[2 * k + (end ? 1 : 0)]);
    if (ev == nullptr) return;
    // while the stream is being captured into a graph, record the event as an
    // external node so each replay records it
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, st);
}
}  // namespace tvlp

using namespace tvlp;

namespace {

constexpr int kMaxDevicesApi = 64;

// Padded orders compiled into the library.
int pad_order(int M, int dtype) {
    if (M <= 0) return 0;
    if (dtype == LP_DTYPE_F32) {
        static const int mp[] = {2, 4, 8, 12, 16, 22, 30, 32};
        for (int v : mp)
            if (M <= v) return v;
    } else if (dtype == LP_DTYPE_F64) {
        static const int mp[] = {2, 4, 8, 12, 16};
        for (int v : mp)
            if (M <= v) return v;
    }
    return -1;
}

template <typename S> struct Dispatch;

#define TVLP_CASE(MPV, CALL) \
    case MPV:                \
        return Impl<S, MPV>::CALL;

template <> struct Dispatch<float> {
    using S = float;
    static Shape shape(int MP) {
        switch (MP) {
            TVLP_CASE(2, shape()) TVLP_CASE(4, shape()) TVLP_CASE(8, shape()) TVLP_CASE(12, shape())
            TVLP_CASE(16, shape()) TVLP_CASE(22, shape()) TVLP_CASE(30, shape()) TVLP_CASE(32, shape())
        }
        return Shape{};
    }
    static int forward(const Problem &p, const S *a, const S *e, const S *zi, S *s, S *ck, int algo, void *ws,
                       cudaStream_t st) {
        switch (p.MP) {
            TVLP_CASE(2, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(4, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(8, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(12, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(16, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(22, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(30, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(32, forward(p, a, e, zi, s, ck, algo, ws, st))
        }
        return EUNSUPPORTED;
    }
    static int rerun(const Problem &p, const S *a, const S *e, const S *ck, const S *zi, S *s, void *ws,
                     cudaStream_t st) {
        switch (p.MP) {
            TVLP_CASE(2, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(4, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(8, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(12, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(16, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(22, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(30, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(32, rerun(p, a, e, ck, zi, s, ws, st))
        }
        return EUNSUPPORTED;
    }
    static int backward(const Problem &p, const S *gs, const S *a, const S *s, const S *zi, S *ge, S *ga, S *gzi,
                        int algo, int flags, void *ws, cudaStream_t st) {
        switch (p.MP) {
            TVLP_CASE(2, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(4, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(8, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(12, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(16, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(22, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(30, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(32, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
        }
        return EUNSUPPORTED;
    }
#define TVLP_ALL_F32(CALL)                                                                            \
    switch (p.MP) {                                                                                   \
        TVLP_CASE(2, CALL) TVLP_CASE(4, CALL) TVLP_CASE(8, CALL) TVLP_CASE(12, CALL) TVLP_CASE(16, CALL) \
        TVLP_CASE(22, CALL) TVLP_CASE(30, CALL) TVLP_CASE(32, CALL)                                   \
    }                                                                                                 \
    return EUNSUPPORTED;
    static int forward_gen(const Problem &p, const CoefSrc &src, const S *e, const S *zi, S *s, S *ck, void *ws,
                           cudaStream_t st) {
        TVLP_ALL_F32(forward_gen(p, src, e, zi, s, ck, ws, st))
    }
    static int backward_gen(const Problem &p, const CoefSrc &src, const S *gs, const S *s, const S *zi, S *ge,
                            S *gzi, int flags, void *ws, cudaStream_t st) {
        TVLP_ALL_F32(backward_gen(p, src, gs, s, zi, ge, gzi, flags, ws, st))
    }
    static int grad_src(const Problem &p, const CoefSrc &src, const S *ge, const S *s, const S *zi, S *gk,
                        void *scratch, cudaStream_t st) {
        TVLP_ALL_F32(grad_src(p, src, ge, s, zi, gk, scratch, st))
    }
#undef TVLP_ALL_F32
};

template <> struct Dispatch<double> {
    using S = double;
    static Shape shape(int MP) {
        switch (MP) {
            TVLP_CASE(2, shape()) TVLP_CASE(4, shape()) TVLP_CASE(8, shape()) TVLP_CASE(12, shape())
            TVLP_CASE(16, shape())
        }
        return Shape{};
    }
    static int forward(const Problem &p, const S *a, const S *e, const S *zi, S *s, S *ck, int algo, void *ws,
                       cudaStream_t st) {
        switch (p.MP) {
            TVLP_CASE(2, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(4, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(8, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(12, forward(p, a, e, zi, s, ck, algo, ws, st))
            TVLP_CASE(16, forward(p, a, e, zi, s, ck, algo, ws, st))
        }
        return EUNSUPPORTED;
    }
    static int rerun(const Problem &p, const S *a, const S *e, const S *ck, const S *zi, S *s, void *ws,
                     cudaStream_t st) {
        switch (p.MP) {
            TVLP_CASE(2, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(4, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(8, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(12, rerun(p, a, e, ck, zi, s, ws, st))
            TVLP_CASE(16, rerun(p, a, e, ck, zi, s, ws, st))
        }
        return EUNSUPPORTED;
    }
    static int backward(const Problem &p, const S *gs, const S *a, const S *s, const S *zi, S *ge, S *ga, S *gzi,
                        int algo, int flags, void *ws, cudaStream_t st) {
        switch (p.MP) {
            TVLP_CASE(2, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(4, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(8, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(12, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
            TVLP_CASE(16, backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st))
        }
        return EUNSUPPORTED;
    }
};
#undef TVLP_CASE

// Per-device lookups cached on first use.  Host threads may make their first
// calls at the same time: the cache entries are atomics, and a lookup done
// twice stores the same value.
int num_sms() {
    static std::atomic<int> cached[kMaxDevicesApi] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesApi) {
        cudaGetLastError();
        return 152;
    }
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

int *status_word() {
    static std::atomic<int *> cached[kMaxDevicesApi] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesApi) {
        cudaGetLastError();
        return nullptr;
    }
    int *w = cached[dev].load(std::memory_order_relaxed);
    if (w == nullptr) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_tvlp_status) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        w = static_cast<int *>(ptr);
        cached[dev].store(w, std::memory_order_relaxed);
    }
    return w;
}

Shape shape_for(int MP, int dtype) {
    return dtype == LP_DTYPE_F32 ? Dispatch<float>::shape(MP) : Dispatch<double>::shape(MP);
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// smallest r with r * r >= x (x >= 0)
int64_t isqrt_ceil(int64_t x) {
    if (x <= 0) return 0;
    int64_t r = (int64_t)std::sqrt((double)x);
    while (r * r < x) ++r;
    while (r > 0 && (r - 1) * (r - 1) >= x) --r;
    return r;
}

// Rough cost model (cycles) of the chunked scan for chunk length L:
// summaries run in waves of resident blocks, each chunk costing L steps; the
// two-level scan costs its group compositions and hops; the re-run is L
// sequential steps.
int pick_chunk_impl(int B, int64_t T, int MP, int dtype) {
    constexpr int SRV = 16;  // chunk lengths are multiples of the stage height
    if (T <= 0 || B <= 0) return SRV;
    const Shape sh = shape_for(MP, dtype);
    const int64_t per_wave = (int64_t)num_sms() * sh.warps_per_block * sh.chunks_per_warp;
    const int64_t max_nblk = ceil_div(T, SRV);
    double best = 1e300;
    int best_L = SRV;
    for (int64_t nblk = 1; nblk <= max_nblk; ++nblk) {
        const int64_t L = nblk * SRV;
        if (L > INT_MAX / 2) break;
        const int64_t nC = ceil_div(T, L);
        const int64_t NQ = (int64_t)B * nC;
        const int64_t waves = ceil_div(NQ, per_wave);
        // two-level scan: G2 compositions and hops, nC / G2 group hops
        int64_t G2 = 1;
        while (G2 * G2 * 4 < nC) ++G2;
        const double scan = (double)G2 * (8.0 * MP * MP / 2 + 300.0) + (double)ceil_div(nC, G2) * 150.0 + 3 * 3000.0;
        const double cost = (double)waves * L * sh.per_step_cycles + scan + (double)L * 40.0;
        if (cost < best) {
            best = cost;
            best_L = (int)L;
        }
    }
    return best_L;
}

bool valid_shape(int B, int64_t T, int M) { return B >= 0 && T >= 0 && M >= 0; }

// Fill a Problem; returns LP_OK or an error code.
int make_problem(int B, int64_t T, int M, int chunk, int dtype, Problem *p) {
    if (!valid_shape(B, T, M)) return LP_EINVAL;
    if (chunk < 0) return LP_EINVAL;
    if (T >= (int64_t)INT_MAX / 2) return LP_EUNSUPPORTED;
    const int MP = pad_order(M, dtype);
    if (M > 0 && MP < 0) return LP_EUNSUPPORTED;
    p->B = B;
    p->T = T;
    p->M = M;
    p->MP = MP;
    p->status = nullptr;
    p->off = nullptr;
    p->items = 0;
    if (M == 0) {
        p->L = 0;
        p->nC = 0;
        p->NQ = 0;
        p->G2 = 1;
        p->nG = 0;
        return LP_OK;
    }
    int L = chunk > 0 ? chunk : pick_chunk_impl(B, T, MP, dtype);
    L = (int)(ceil_div(L, 16) * 16);
    if (L <= 0) return LP_EINVAL;
    p->L = L;
    p->nC = T > 0 ? ceil_div(T, L) : 0;
    p->NQ = (int64_t)B * p->nC;
    // two-level scan: groups of about sqrt(nC / 4) chunks
    int64_t G2 = 1;
    while (G2 * G2 * 4 < p->nC) ++G2;
    p->G2 = (int)G2;
    p->nG = (int)ceil_div(p->nC > 0 ? p->nC : 1, G2);
    p->items = (int64_t)B * p->nG;
    return LP_OK;
}

// Varlen batch: n signals packed back to back, total rows in all, at device
// offsets `off` [n+1].  Chunk and group counts are upper bounds (each signal
// adds at most one partial chunk); the kernels read the exact ones from the
// tables built at the start of every call.
int make_problem_varlen(int n, int64_t total, int M, int chunk, int dtype, const int64_t *off, Problem *p) {
    if (n < 0 || total < 0 || M < 0 || chunk < 0) return LP_EINVAL;
    if (total >= (int64_t)INT_MAX / 2) return LP_EUNSUPPORTED;
    const int MP = pad_order(M, dtype);
    if (M > 0 && MP < 0) return LP_EUNSUPPORTED;
    p->B = n;
    p->T = total;
    p->M = M;
    p->MP = MP;
    p->status = nullptr;
    p->off = off;
    p->nC = 0;
    p->G2 = 0;
    p->nG = 0;
    if (M == 0 || n == 0) {
        p->L = 0;
        p->NQ = 0;
        p->items = 0;
        return LP_OK;
    }
    int L = chunk > 0 ? chunk : pick_chunk_impl(n, ceil_div(total, n), MP, dtype);
    L = (int)(ceil_div(L, 16) * 16);
    if (L <= 0) return LP_EINVAL;
    p->L = L;
    p->NQ = ceil_div(total, L) + n;
    // scan groups: a signal of c chunks has ceil(c / g) groups of g >=
    // sqrt(c / 4) chunks, at most 2 sqrt(c) + 1; over the batch (sum of c
    // at most NQ) at most 2 sqrt(n NQ) + n by Cauchy-Schwarz
    const int64_t bound = 2 * isqrt_ceil((int64_t)n * p->NQ) + n + 1;
    p->items = bound < p->NQ ? bound : p->NQ;
    return LP_OK;
}

size_t workspace_for(const Problem &p, int dtype) {
    if (p.M == 0 || p.NQ == 0) return 0;
    return ws_bytes(p, dtype == LP_DTYPE_F32 ? 4 : 8);
}

bool aligned(const void *ptr, size_t n) { return (reinterpret_cast<uintptr_t>(ptr) % n) == 0; }

int check_workspace(const Problem &p, int dtype, int algo, const void *ws, size_t bytes) {
    if (algo == LP_ALGO_PLAIN) return LP_OK;
    const size_t need = workspace_for(p, dtype);
    if (need == 0) return LP_OK;
    if (ws == nullptr || bytes < need || !aligned(ws, 256)) return LP_EWORKSPACE;
    return LP_OK;
}

template <typename S>
int forward_impl(int dtype, int B, int64_t T, int M, const S *a, const S *e, const S *zi, S *s, S *ckpt,
                 int chunk, int algo, void *ws, size_t wsb, void *stream) {
    if (algo != LP_ALGO_CHUNKED && algo != LP_ALGO_PLAIN) return LP_EINVAL;
    Problem p;
    int rc = make_problem(B, T, M, chunk, dtype, &p);
    if (rc != LP_OK) return rc;
    if (B == 0 || T == 0) return LP_OK;
    if (e == nullptr || s == nullptr || (M > 0 && a == nullptr)) return LP_EINVAL;
    if (ckpt != nullptr && algo != LP_ALGO_CHUNKED) return LP_EINVAL;
    if (!aligned(e, sizeof(S)) || !aligned(s, sizeof(S)) || !aligned(a, 2 * sizeof(S)) ||
        !aligned(zi, sizeof(S)) || !aligned(ckpt, sizeof(S)))
        return LP_EALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (M == 0) {
        if (cudaMemcpyAsync(s, e, (size_t)B * T * sizeof(S), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if ((rc = check_workspace(p, dtype, algo, ws, wsb)) != LP_OK) return rc;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    return Dispatch<S>::forward(p, a, e, zi, s, ckpt, algo, ws, st);
}

template <typename S>
int backward_impl(int dtype, int B, int64_t T, int M, const S *gs, const S *a, const S *s, const S *zi, S *ge,
                  S *ga, S *gzi, int chunk, int algo, int flags, void *ws, size_t wsb, void *stream) {
    if (algo != LP_ALGO_CHUNKED && algo != LP_ALGO_PLAIN) return LP_EINVAL;
    if ((flags & ~(LP_BWD_REUSE_FORWARD | LP_BWD_FUSED_GA)) != 0) return LP_EINVAL;
    Problem p;
    int rc = make_problem(B, T, M, chunk, dtype, &p);
    if (rc != LP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (B == 0) return LP_OK;
    if (T == 0) {
        // no samples: the initial-state gradient is zero
        if (gzi != nullptr && M > 0 && cudaMemsetAsync(gzi, 0, (size_t)B * M * sizeof(S), st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if (gs == nullptr || ge == nullptr || (M > 0 && a == nullptr) || (ga != nullptr && s == nullptr))
        return LP_EINVAL;
    if (!aligned(gs, sizeof(S)) || !aligned(ge, sizeof(S)) || !aligned(a, 2 * sizeof(S)) ||
        !aligned(s, sizeof(S)) || !aligned(zi, sizeof(S)) || !aligned(ga, sizeof(S)) || !aligned(gzi, sizeof(S)))
        return LP_EALIGN;
    if (M == 0) {
        if (cudaMemcpyAsync(ge, gs, (size_t)B * T * sizeof(S), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if ((rc = check_workspace(p, dtype, algo, ws, wsb)) != LP_OK) return rc;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    return Dispatch<S>::backward(p, gs, a, s, zi, ge, ga, gzi, algo, flags, ws, st);
}


// Backward from chunk checkpoints: s is recomputed into `s` from a, e and the
// forward's per-chunk incoming states, then the adjoint runs as usual.
template <typename S>
int backward_recompute_impl(int dtype, int B, int64_t T, int M, const S *gs, const S *a, const S *e, const S *ckpt,
                            const S *zi, S *s, S *ge, S *ga, S *gzi, int chunk, int flags, void *ws, size_t wsb,
                            void *stream) {
    if ((flags & ~(LP_BWD_REUSE_FORWARD | LP_BWD_FUSED_GA)) != 0) return LP_EINVAL;
    Problem p;
    int rc = make_problem(B, T, M, chunk, dtype, &p);
    if (rc != LP_OK) return rc;
    if (B == 0 || T == 0 || M == 0)  // no recursion: s = e
        return backward_impl<S>(dtype, B, T, M, gs, a, e, zi, ge, ga, gzi, chunk, LP_ALGO_CHUNKED, flags, ws, wsb,
                                stream);
    if (e == nullptr || ckpt == nullptr || s == nullptr || a == nullptr) return LP_EINVAL;
    if (!aligned(e, sizeof(S)) || !aligned(ckpt, sizeof(S)) || !aligned(s, sizeof(S)) || !aligned(a, 2 * sizeof(S)))
        return LP_EALIGN;
    if ((rc = check_workspace(p, dtype, LP_ALGO_CHUNKED, ws, wsb)) != LP_OK) return rc;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    if ((rc = Dispatch<S>::rerun(p, a, e, ckpt, zi, s, ws, static_cast<cudaStream_t>(stream))) != LP_OK) return rc;
    return backward_impl<S>(dtype, B, T, M, gs, a, s, zi, ge, ga, gzi, chunk, LP_ALGO_CHUNKED, flags, ws, wsb,
                            stream);
}


template <typename S>
int forward_varlen_impl(int dtype, int n, const int64_t *off, int64_t total, int M, const S *a, const S *e,
                        const S *zi, S *s, S *ckpt, int chunk, void *ws, size_t wsb, void *stream) {
    Problem p;
    int rc = make_problem_varlen(n, total, M, chunk, dtype, off, &p);
    if (rc != LP_OK) return rc;
    if (n == 0 || total == 0) return LP_OK;
    if (off == nullptr || e == nullptr || s == nullptr || (M > 0 && a == nullptr)) return LP_EINVAL;
    if (!aligned(off, 8) || !aligned(e, sizeof(S)) || !aligned(s, sizeof(S)) || !aligned(a, 2 * sizeof(S)) ||
        !aligned(zi, sizeof(S)) || !aligned(ckpt, sizeof(S)))
        return LP_EALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (M == 0) {
        if (cudaMemcpyAsync(s, e, (size_t)total * sizeof(S), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if ((rc = check_workspace(p, dtype, LP_ALGO_CHUNKED, ws, wsb)) != LP_OK) return rc;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    return Dispatch<S>::forward(p, a, e, zi, s, ckpt, LP_ALGO_CHUNKED, ws, st);
}

template <typename S>
int backward_varlen_impl(int dtype, int n, const int64_t *off, int64_t total, int M, const S *gs, const S *a,
                         const S *s, const S *zi, S *ge, S *ga, S *gzi, int chunk, int flags, void *ws, size_t wsb,
                         void *stream) {
    if ((flags & ~(LP_BWD_REUSE_FORWARD | LP_BWD_FUSED_GA)) != 0) return LP_EINVAL;
    Problem p;
    int rc = make_problem_varlen(n, total, M, chunk, dtype, off, &p);
    if (rc != LP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return LP_OK;
    if (total == 0) {
        if (gzi != nullptr && M > 0 && cudaMemsetAsync(gzi, 0, (size_t)n * M * sizeof(S), st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if (off == nullptr || gs == nullptr || ge == nullptr || (M > 0 && a == nullptr) || (ga != nullptr && s == nullptr))
        return LP_EINVAL;
    if (!aligned(off, 8) || !aligned(gs, sizeof(S)) || !aligned(ge, sizeof(S)) || !aligned(a, 2 * sizeof(S)) ||
        !aligned(s, sizeof(S)) || !aligned(zi, sizeof(S)) || !aligned(ga, sizeof(S)) || !aligned(gzi, sizeof(S)))
        return LP_EALIGN;
    if (M == 0) {
        if (cudaMemcpyAsync(ge, gs, (size_t)total * sizeof(S), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if ((rc = check_workspace(p, dtype, LP_ALGO_CHUNKED, ws, wsb)) != LP_OK) return rc;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    // empty signals have no first chunk to write their (zero) gzi
    if (gzi != nullptr && cudaMemsetAsync(gzi, 0, (size_t)n * M * sizeof(S), st) != cudaSuccess) return LP_ECUDA;
    return Dispatch<S>::backward(p, gs, a, s, zi, ge, ga, gzi, LP_ALGO_CHUNKED, flags, ws, st);
}


// ---------------------------------------------------------------------------
// Generated coefficients: time-invariant rows (SRC_CONST) and frame-rate
// reflection coefficients (SRC_FRAMES).  FP32, chunked.
// ---------------------------------------------------------------------------
int64_t frames_of(int64_t T, int hop) { return ceil_div(T, hop) + 1; }

// scratch of the coefficient gradient, after the scan workspace
size_t grad_scratch_bytes(const Problem &p, int kind, int64_t F) {
    if (p.M == 0 || p.T == 0 || p.B == 0) return 0;
    if (kind == SRC_CONST) return align256((size_t)p.B * (size_t)ceil_div(p.T, 1024) * p.MP * sizeof(float));
    return align256(2 * (size_t)p.B * (size_t)F * p.M * sizeof(float));
}

size_t gen_workspace_bytes(const Problem &p, int kind, int64_t F) {
    return align256(workspace_for(p, LP_DTYPE_F32)) + grad_scratch_bytes(p, kind, F);
}

// frames, M one of the compiled orders: the generated-row cache after the
// gradient's scratch (0: no cache for this problem)
size_t row_cache_bytes(const Problem &p, int kind) {
    if (kind != SRC_FRAMES || p.M != p.MP || p.M == 0) return 0;
    return align256((size_t)p.B * (size_t)p.T * p.MP * sizeof(float));
}
float *row_cache(const Problem &p, int kind, int64_t F, void *ws, size_t wsb) {
    const size_t off = gen_workspace_bytes(p, kind, F), n = row_cache_bytes(p, kind);
    if (n == 0 || wsb < off + n) return nullptr;
    return reinterpret_cast<float *>(static_cast<char *>(ws) + off);
}

// Varlen frames, M one of the compiled orders: the generated-row cache
// ([total][MP]) starts right after the scan workspace.  The varlen forward
// does not know the frame count, so here the gradient's scratch follows the
// cache (when the workspace holds both) instead of preceding it.
size_t varlen_cache_bytes(const Problem &p) {
    if (p.M != p.MP || p.M == 0) return 0;
    return align256((size_t)p.T * p.MP * sizeof(float));  // p.T: packed rows
}

CoefSrc make_src(int kind, const float *k, int64_t F, int hop) {
    CoefSrc c;
    c.kind = kind;
    c.k = k;
    c.F = F;
    c.hop = hop > 0 ? hop : 1;
    c.inv_hop = 1.0f / (float)c.hop;
    return c;
}

int forward_gen_impl(int kind, int B, int64_t T, int M, int hop, const float *k, const float *e, const float *zi,
                     float *s, float *ckpt, int chunk, void *ws, size_t wsb, void *stream) {
    if (kind == SRC_FRAMES && hop < 1) return LP_EINVAL;
    Problem p;
    int rc = make_problem(B, T, M, chunk, LP_DTYPE_F32, &p);
    if (rc != LP_OK) return rc;
    if (B == 0 || T == 0) return LP_OK;
    if (e == nullptr || s == nullptr || (M > 0 && k == nullptr)) return LP_EINVAL;
    if (!aligned(e, 4) || !aligned(s, 4) || !aligned(k, 4) || !aligned(zi, 4) || !aligned(ckpt, 4)) return LP_EALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (M == 0) {
        if (cudaMemcpyAsync(s, e, (size_t)B * T * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    const int64_t F = kind == SRC_FRAMES ? frames_of(T, hop) : 1;
    if (ws == nullptr || !aligned(ws, 256) || wsb < workspace_for(p, LP_DTYPE_F32)) return LP_EWORKSPACE;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    CoefSrc src = make_src(kind, k, F, hop);
    src.cache = row_cache(p, kind, F, ws, wsb);
    return Dispatch<float>::forward_gen(p, src, e, zi, s, ckpt, ws, st);
}

int backward_gen_impl(int kind, int B, int64_t T, int M, int hop, const float *gs, const float *k, const float *s,
                      const float *zi, float *ge, float *gk, float *gzi, int chunk, int flags, void *ws, size_t wsb,
                      void *stream) {
    if (kind == SRC_FRAMES && hop < 1) return LP_EINVAL;
    if ((flags & ~LP_BWD_REUSE_FORWARD) != 0) return LP_EINVAL;
    Problem p;
    int rc = make_problem(B, T, M, chunk, LP_DTYPE_F32, &p);
    if (rc != LP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (B == 0 || (M == 0 && T == 0)) return LP_OK;
    const int64_t F = kind == SRC_FRAMES ? frames_of(T, hop) : 1;
    if (T == 0) {
        // no samples: every gradient is zero
        if (gzi != nullptr && cudaMemsetAsync(gzi, 0, (size_t)B * M * sizeof(float), st) != cudaSuccess)
            return LP_ECUDA;
        if (gk != nullptr && cudaMemsetAsync(gk, 0, (size_t)B * F * M * sizeof(float), st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if (gs == nullptr || ge == nullptr || (M > 0 && k == nullptr) || (gk != nullptr && s == nullptr))
        return LP_EINVAL;
    if (!aligned(gs, 4) || !aligned(ge, 4) || !aligned(k, 4) || !aligned(s, 4) || !aligned(zi, 4) ||
        !aligned(gk, 4) || !aligned(gzi, 4))
        return LP_EALIGN;
    if (M == 0) {
        if (cudaMemcpyAsync(ge, gs, (size_t)B * T * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if (ws == nullptr || !aligned(ws, 256) || wsb < (gk != nullptr ? gen_workspace_bytes(p, kind, F)
                                                                    : workspace_for(p, LP_DTYPE_F32)))
        return LP_EWORKSPACE;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    CoefSrc src = make_src(kind, k, F, hop);
    // the rows the forward cached in this workspace (used with
    // LP_BWD_REUSE_FORWARD only)
    src.cache = row_cache(p, kind, F, ws, wsb);
    if ((rc = Dispatch<float>::backward_gen(p, src, gs, s, zi, ge, gzi, flags, ws, st)) != LP_OK) return rc;
    if (gk == nullptr) return LP_OK;
    void *scratch = static_cast<char *>(ws) + align256(workspace_for(p, LP_DTYPE_F32));
    return Dispatch<float>::grad_src(p, src, ge, s, zi, gk, scratch, st);
}

int forward_frames_varlen_impl(int n, const int64_t *off, int64_t total, int M, int hop, const int64_t *foff,
                               const float *k, const float *e, const float *zi, float *s, float *ckpt, int chunk,
                               void *ws, size_t wsb, void *stream) {
    if (hop < 1) return LP_EINVAL;
    Problem p;
    int rc = make_problem_varlen(n, total, M, chunk, LP_DTYPE_F32, off, &p);
    if (rc != LP_OK) return rc;
    if (n == 0 || total == 0) return LP_OK;
    if (off == nullptr || e == nullptr || s == nullptr || (M > 0 && (k == nullptr || foff == nullptr)))
        return LP_EINVAL;
    if (!aligned(off, 8) || !aligned(foff, 8) || !aligned(e, 4) || !aligned(s, 4) || !aligned(k, 4) ||
        !aligned(zi, 4) || !aligned(ckpt, 4))
        return LP_EALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (M == 0) {
        if (cudaMemcpyAsync(s, e, (size_t)total * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if ((rc = check_workspace(p, LP_DTYPE_F32, LP_ALGO_CHUNKED, ws, wsb)) != LP_OK) return rc;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    CoefSrc src = make_src(SRC_FRAMES, k, 0, hop);
    src.foff = foff;
    const size_t base = align256(workspace_for(p, LP_DTYPE_F32)), cb = varlen_cache_bytes(p);
    if (cb > 0 && wsb >= base + cb) src.cache = reinterpret_cast<float *>(static_cast<char *>(ws) + base);
    return Dispatch<float>::forward_gen(p, src, e, zi, s, ckpt, ws, st);
}

// Varlen adjoint with frames: gk has total_frames rows (the packed frames).
size_t frames_varlen_workspace_bytes(const Problem &p, int64_t total_frames) {
    return align256(workspace_for(p, LP_DTYPE_F32)) + align256(2 * (size_t)total_frames * p.M * sizeof(float));
}

int backward_frames_varlen_impl(int n, const int64_t *off, int64_t total, int M, int hop, const int64_t *foff,
                                int64_t total_frames, const float *gs, const float *k, const float *s,
                                const float *zi, float *ge, float *gk, float *gzi, int chunk, int flags, void *ws,
                                size_t wsb, void *stream) {
    if (hop < 1 || total_frames < 0) return LP_EINVAL;
    if ((flags & ~LP_BWD_REUSE_FORWARD) != 0) return LP_EINVAL;
    Problem p;
    int rc = make_problem_varlen(n, total, M, chunk, LP_DTYPE_F32, off, &p);
    if (rc != LP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return LP_OK;
    if (total == 0 || M == 0) {
        if (gzi != nullptr && M > 0 && cudaMemsetAsync(gzi, 0, (size_t)n * M * sizeof(float), st) != cudaSuccess)
            return LP_ECUDA;
        if (gk != nullptr && M > 0 &&
            cudaMemsetAsync(gk, 0, (size_t)total_frames * M * sizeof(float), st) != cudaSuccess)
            return LP_ECUDA;
        if (M == 0 && total > 0 &&
            cudaMemcpyAsync(ge, gs, (size_t)total * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return LP_ECUDA;
        return LP_OK;
    }
    if (off == nullptr || foff == nullptr || gs == nullptr || ge == nullptr || k == nullptr ||
        (gk != nullptr && s == nullptr))
        return LP_EINVAL;
    if (!aligned(off, 8) || !aligned(foff, 8) || !aligned(gs, 4) || !aligned(ge, 4) || !aligned(k, 4) ||
        !aligned(s, 4) || !aligned(zi, 4) || !aligned(gk, 4) || !aligned(gzi, 4))
        return LP_EALIGN;
    const size_t need = gk != nullptr ? frames_varlen_workspace_bytes(p, total_frames) : workspace_for(p, LP_DTYPE_F32);
    if (ws == nullptr || !aligned(ws, 256) || wsb < need) return LP_EWORKSPACE;
    if ((p.status = status_word()) == nullptr) return LP_ECUDA;
    CoefSrc src = make_src(SRC_FRAMES, k, total_frames, hop);
    src.foff = foff;
    // empty signals have no chunk to write their (zero) gzi
    if (gzi != nullptr && cudaMemsetAsync(gzi, 0, (size_t)n * M * sizeof(float), st) != cudaSuccess) return LP_ECUDA;
    // the forward's cached rows, when the workspace holds them and the
    // gradient's scratch after them
    const size_t base = align256(workspace_for(p, LP_DTYPE_F32)), cb = varlen_cache_bytes(p);
    const size_t sb = gk != nullptr ? align256(2 * (size_t)total_frames * p.M * sizeof(float)) : 0;
    const bool cached = cb > 0 && (flags & LP_BWD_REUSE_FORWARD) && wsb >= base + cb + sb;
    if (cached) src.cache = reinterpret_cast<float *>(static_cast<char *>(ws) + base);
    if ((rc = Dispatch<float>::backward_gen(p, src, gs, s, zi, ge, gzi, flags, ws, st)) != LP_OK) return rc;
    if (gk == nullptr) return LP_OK;
    void *scratch = static_cast<char *>(ws) + base + (cached ? cb : 0);
    return Dispatch<float>::grad_src(p, src, ge, s, zi, gk, scratch, st);
}
}  // namespace

// The device status word of the current device, for the other translation
// units of the library (nullptr if unavailable).
int *tvlp::device_status_word() { return status_word(); }

extern "C" {

const char *lp_strerror(int code) {
    switch (code) {
        case LP_OK: return "ok";
        case LP_EINVAL: return "invalid argument (shape, NULL pointer or flag)";
        case LP_EUNSUPPORTED: return "unsupported order or length for this build";
        case LP_EWORKSPACE: return "workspace missing, too small or not 256-byte aligned";
        case LP_ECUDA: return "CUDA launch or runtime call failed";
        case LP_EALIGN: return "data pointer not aligned to its element type";
        case LP_ETOOBIG: return "problem needs more scratch than the fixed no-allocation array holds";
        case LP_ETIMEOUT: return "a bounded wait ended before its condition held";
        case LP_ENONFINITE: return "an infinity or NaN was found";
    }
    return "unknown error code";
}

const char *lp_version(void) { return "tvlp 0.1 sm_103a"; }

int lp_tv_set_threads_per_chunk(int k1_lane_factor, int rerun_chunks_per_warp) {
    if (k1_lane_factor == 0) k1_lane_factor = 1;
    if (rerun_chunks_per_warp == 0) rerun_chunks_per_warp = 16;
    if ((k1_lane_factor != 1 && k1_lane_factor != 2) || (rerun_chunks_per_warp != 16 && rerun_chunks_per_warp != 8))
        return LP_EINVAL;
    g_shape.k1_lane_factor = k1_lane_factor;
    g_shape.rec_chunks = rerun_chunks_per_warp;
    return LP_OK;
}

int lp_tv_set_profile_events(void **events, int n) {
    if (events != nullptr && n < 0) return LP_EINVAL;
    g_prof_events = events;
    g_prof_n = events ? n : 0;
    return LP_OK;
}

int lp_tv_pick_chunk(int B, int64_t T, int M, int dtype) {
    Problem p;
    if (make_problem(B, T, M, 0, dtype, &p) != LP_OK) return 0;
    return p.L;
}

int64_t lp_tv_num_chunks(int64_t T, int M, int chunk) {
    if (T <= 0 || M <= 0 || chunk <= 0) return 0;
    const int64_t L = ceil_div(chunk, 16) * 16;
    return ceil_div(T, L);
}

size_t lp_tv_workspace_bytes(int B, int64_t T, int M, int chunk, int dtype) {
    if (dtype != LP_DTYPE_F32 && dtype != LP_DTYPE_F64) return 0;
    Problem p;
    if (make_problem(B, T, M, chunk, dtype, &p) != LP_OK) return 0;
    return workspace_for(p, dtype);
}

int lp_tv_forward_f32(int B, int64_t T, int M, const float *a, const float *e, const float *zi, float *s,
                      float *ckpt, int chunk, int algo, void *workspace, size_t workspace_bytes, void *stream) {
    return forward_impl<float>(LP_DTYPE_F32, B, T, M, a, e, zi, s, ckpt, chunk, algo, workspace, workspace_bytes,
                               stream);
}

int lp_tv_forward_f64(int B, int64_t T, int M, const double *a, const double *e, const double *zi, double *s,
                      double *ckpt, int chunk, int algo, void *workspace, size_t workspace_bytes, void *stream) {
    return forward_impl<double>(LP_DTYPE_F64, B, T, M, a, e, zi, s, ckpt, chunk, algo, workspace,
                                workspace_bytes, stream);
}

int lp_tv_backward_f32(int B, int64_t T, int M, const float *gs, const float *a, const float *s, const float *zi,
                       float *ge, float *ga, float *gzi, int chunk, int algo, int flags, void *workspace,
                       size_t workspace_bytes, void *stream) {
    return backward_impl<float>(LP_DTYPE_F32, B, T, M, gs, a, s, zi, ge, ga, gzi, chunk, algo, flags, workspace,
                                workspace_bytes, stream);
}

int lp_tv_backward_f64(int B, int64_t T, int M, const double *gs, const double *a, const double *s,
                       const double *zi, double *ge, double *ga, double *gzi, int chunk, int algo, int flags,
                       void *workspace, size_t workspace_bytes, void *stream) {
    return backward_impl<double>(LP_DTYPE_F64, B, T, M, gs, a, s, zi, ge, ga, gzi, chunk, algo, flags, workspace,
                                 workspace_bytes, stream);
}

int lp_tv_device_status(int reset) {
    int *w = status_word();
    if (w == nullptr) return LP_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LP_ECUDA;
    if (reset && v != 0) {
        const int zero = 0;
        if (cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return LP_ECUDA;
    }
    return v;
}

int lp_tv_backward_recompute_f32(int B, int64_t T, int M, const float *gs, const float *a, const float *e,
                                 const float *ckpt, const float *zi, float *s, float *ge, float *ga, float *gzi,
                                 int chunk, int flags, void *workspace, size_t workspace_bytes, void *stream) {
    return backward_recompute_impl<float>(LP_DTYPE_F32, B, T, M, gs, a, e, ckpt, zi, s, ge, ga, gzi, chunk, flags,
                                          workspace, workspace_bytes, stream);
}

int lp_tv_backward_recompute_f64(int B, int64_t T, int M, const double *gs, const double *a, const double *e,
                                 const double *ckpt, const double *zi, double *s, double *ge, double *ga,
                                 double *gzi, int chunk, int flags, void *workspace, size_t workspace_bytes,
                                 void *stream) {
    return backward_recompute_impl<double>(LP_DTYPE_F64, B, T, M, gs, a, e, ckpt, zi, s, ge, ga, gzi, chunk, flags,
                                           workspace, workspace_bytes, stream);
}

size_t lp_tv_workspace_bytes_varlen(int n, int64_t total, int M, int chunk, int dtype) {
    if (dtype != LP_DTYPE_F32 && dtype != LP_DTYPE_F64) return 0;
    Problem p;
    if (make_problem_varlen(n, total, M, chunk, dtype, nullptr, &p) != LP_OK) return 0;
    p.off = reinterpret_cast<const int64_t *>(1);  // size the tables region too
    return workspace_for(p, dtype);
}

int lp_tv_forward_varlen_f32(int n, const int64_t *offsets, int64_t total, int M, const float *a, const float *e,
                             const float *zi, float *s, float *ckpt, int chunk, void *workspace,
                             size_t workspace_bytes, void *stream) {
    return forward_varlen_impl<float>(LP_DTYPE_F32, n, offsets, total, M, a, e, zi, s, ckpt, chunk, workspace,
                                      workspace_bytes, stream);
}

int lp_tv_forward_varlen_f64(int n, const int64_t *offsets, int64_t total, int M, const double *a, const double *e,
                             const double *zi, double *s, double *ckpt, int chunk, void *workspace,
                             size_t workspace_bytes, void *stream) {
    return forward_varlen_impl<double>(LP_DTYPE_F64, n, offsets, total, M, a, e, zi, s, ckpt, chunk, workspace,
                                       workspace_bytes, stream);
}

int lp_tv_backward_varlen_f32(int n, const int64_t *offsets, int64_t total, int M, const float *gs, const float *a,
                              const float *s, const float *zi, float *ge, float *ga, float *gzi, int chunk,
                              int flags, void *workspace, size_t workspace_bytes, void *stream) {
    return backward_varlen_impl<float>(LP_DTYPE_F32, n, offsets, total, M, gs, a, s, zi, ge, ga, gzi, chunk, flags,
                                       workspace, workspace_bytes, stream);
}

int lp_tv_backward_varlen_f64(int n, const int64_t *offsets, int64_t total, int M, const double *gs,
                              const double *a, const double *s, const double *zi, double *ge, double *ga,
                              double *gzi, int chunk, int flags, void *workspace, size_t workspace_bytes,
                              void *stream) {
    return backward_varlen_impl<double>(LP_DTYPE_F64, n, offsets, total, M, gs, a, s, zi, ge, ga, gzi, chunk, flags,
                                        workspace, workspace_bytes, stream);
}

size_t lp_tv_workspace_bytes_frames(int B, int64_t T, int M, int hop, int chunk) {
    Problem p;
    if (hop < 1 || make_problem(B, T, M, chunk, LP_DTYPE_F32, &p) != LP_OK) return 0;
    return gen_workspace_bytes(p, SRC_FRAMES, frames_of(T, hop));
}

size_t lp_tv_workspace_bytes_frames_cached(int B, int64_t T, int M, int hop, int chunk) {
    Problem p;
    if (hop < 1 || make_problem(B, T, M, chunk, LP_DTYPE_F32, &p) != LP_OK) return 0;
    return gen_workspace_bytes(p, SRC_FRAMES, frames_of(T, hop)) + row_cache_bytes(p, SRC_FRAMES);
}

int lp_tv_forward_frames_f32(int B, int64_t T, int M, int hop, const float *k, const float *e, const float *zi,
                             float *s, float *ckpt, int chunk, void *ws, size_t wsb, void *stream) {
    return forward_gen_impl(SRC_FRAMES, B, T, M, hop, k, e, zi, s, ckpt, chunk, ws, wsb, stream);
}

int lp_tv_backward_frames_f32(int B, int64_t T, int M, int hop, const float *gs, const float *k, const float *s,
                              const float *zi, float *ge, float *gk, float *gzi, int chunk, int flags, void *ws,
                              size_t wsb, void *stream) {
    return backward_gen_impl(SRC_FRAMES, B, T, M, hop, gs, k, s, zi, ge, gk, gzi, chunk, flags, ws, wsb, stream);
}

int lp_tv_forward_frames_varlen_f32(int n, const int64_t *offsets, int64_t total, int M, int hop,
                                    const int64_t *frame_offsets, const float *k, const float *e, const float *zi,
                                    float *s, float *ckpt, int chunk, void *ws, size_t wsb, void *stream) {
    return forward_frames_varlen_impl(n, offsets, total, M, hop, frame_offsets, k, e, zi, s, ckpt, chunk, ws, wsb,
                                      stream);
}

size_t lp_tv_workspace_bytes_ti(int B, int64_t T, int M, int chunk) {
    Problem p;
    if (make_problem(B, T, M, chunk, LP_DTYPE_F32, &p) != LP_OK) return 0;
    return gen_workspace_bytes(p, SRC_CONST, 1);
}

int lp_tv_forward_ti_f32(int B, int64_t T, int M, const float *a, const float *e, const float *zi, float *s,
                         float *ckpt, int chunk, void *ws, size_t wsb, void *stream) {
    return forward_gen_impl(SRC_CONST, B, T, M, 0, a, e, zi, s, ckpt, chunk, ws, wsb, stream);
}

int lp_tv_backward_ti_f32(int B, int64_t T, int M, const float *gs, const float *a, const float *s, const float *zi,
                          float *ge, float *ga, float *gzi, int chunk, int flags, void *ws, size_t wsb,
                          void *stream) {
    return backward_gen_impl(SRC_CONST, B, T, M, 0, gs, a, s, zi, ge, ga, gzi, chunk, flags, ws, wsb, stream);
}

size_t lp_tv_workspace_bytes_frames_varlen(int n, int64_t total, int M, int64_t total_frames, int chunk) {
    Problem p;
    if (total_frames < 0 || make_problem_varlen(n, total, M, chunk, LP_DTYPE_F32, nullptr, &p) != LP_OK) return 0;
    p.off = reinterpret_cast<const int64_t *>(1);  // size the tables region too
    return frames_varlen_workspace_bytes(p, total_frames);
}

size_t lp_tv_workspace_bytes_frames_varlen_cached(int n, int64_t total, int M, int64_t total_frames, int chunk) {
    Problem p;
    if (total_frames < 0 || make_problem_varlen(n, total, M, chunk, LP_DTYPE_F32, nullptr, &p) != LP_OK) return 0;
    p.off = reinterpret_cast<const int64_t *>(1);  // size the tables region too
    return frames_varlen_workspace_bytes(p, total_frames) + varlen_cache_bytes(p);
}

int lp_tv_backward_frames_varlen_f32(int n, const int64_t *offsets, int64_t total, int M, int hop,
                                     const int64_t *frame_offsets, int64_t total_frames, const float *gs,
                                     const float *k, const float *s, const float *zi, float *ge, float *gk,
                                     float *gzi, int chunk, int flags, void *ws, size_t wsb, void *stream) {
    return backward_frames_varlen_impl(n, offsets, total, M, hop, frame_offsets, total_frames, gs, k, s, zi, ge, gk,
                                       gzi, chunk, flags, ws, wsb, stream);
}

int lp_tv_l2_set_aside(size_t bytes, size_t *applied) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LP_ECUDA;
    int max_bytes = 0;
    if (cudaDeviceGetAttribute(&max_bytes, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess) return LP_ECUDA;
    const size_t want = bytes > (size_t)max_bytes ? (size_t)max_bytes : bytes;
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) return LP_ECUDA;
    size_t got = 0;
    if (cudaDeviceGetLimit(&got, cudaLimitPersistingL2CacheSize) != cudaSuccess) return LP_ECUDA;
    if (applied != nullptr) *applied = got;
    return LP_OK;
}

}  // extern "C"
