// Host launchers of the time-varying LP kernels for one (scalar, MP) pair.
#pragma once
#include <atomic>

#include "tvlp_impl.h"
#include "tvlp_kernels.cuh"

namespace tvlp {

constexpr size_t kSmemBudget = 200 * 1024;  // dynamic shared memory per K1 block
constexpr size_t kL2Keep = 80u << 20;        // bytes of `a` a pass keeps in L2 for the next
constexpr int kMaxDevices = 64;

template <typename S, int MP> using DefaultSumGeo = SumGeo<S, MP, Pack<MP>::G, Pack<MP>::R>;

template <typename S, int MP> using WideSumGeo = SumGeo<S, MP, PackWide<MP>::G, PackWide<MP>::R>;

template <typename GE> inline int k1_warps_for() {
    int w = (int)(kSmemBudget / GE::WARP_BYTES);
    return w > 8 ? 8 : (w < 1 ? 1 : w);
}
template <typename S, int MP> inline int k1_warps_per_block() { return k1_warps_for<DefaultSumGeo<S, MP>>(); }

// Launch with programmatic stream serialization (the kernel may start while
// the previous kernel on the stream finishes; see pdl_wait in the kernels),
// optionally as a cooperative launch (all blocks resident).
template <typename... Exp, typename... Act>
inline cudaError_t launch(void (*kern)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool coop,
                          Act &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int n = 0;
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
    if (coop) {
        attr[n].id = cudaLaunchAttributeCooperative;
        attr[n].val.cooperative = 1;
        ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Exp>(args)...);
}

// cudaFuncSetAttribute once per kernel and device.  Host threads may race
// on the first call: the flags are atomics, and setting the same attribute
// twice is harmless.
template <typename K> inline cudaError_t allow_smem(K kernel, size_t bytes, std::atomic<bool> *done) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err == cudaSuccess) done[dev].store(true, std::memory_order_release);
    return err;
}

template <typename S, int MP> Shape Impl<S, MP>::shape() {
    using GE = DefaultSumGeo<S, MP>;
    Shape sh;
    sh.chunks_per_warp = GE::CPW;
    sh.warps_per_block = k1_warps_per_block<S, MP>();
    const int wps = (sh.warps_per_block + 3) / 4;  // warps sharing a scheduler
    sh.per_step_cycles = (GE::R * MP + MP / 2 + GE::R * MP / SR + 4) * wps;
    sh.ws_per_chunk = (size_t)(YGeo<S, MP>::YS + 3 * MP) * sizeof(S);
    return sh;
}

// The kernels' view of where a problem's chunks lie.
inline Batch batch_of(const Problem &p, void *ws, size_t sz) {
    Batch bt;
    bt.T = p.T;
    bt.nC = p.nC;
    bt.G2 = p.G2;
    bt.nG = p.nG;
    bt.off = p.off;
    bt.n = p.B;
    bt.cstart = bt.gstart = nullptr;
    bt.sig = bt.ord = nullptr;
    bt.aoff = nullptr;
    bt.ldz = 0;
    if (p.off != nullptr) {
        int *tab = reinterpret_cast<int *>(static_cast<char *>(ws) + ws_offset(p, sz, 8));
        bt.cstart = tab;
        bt.gstart = tab + p.B + 1;
    }
    return bt;
}

template <typename S, int MP> struct Launch {
    using GE = DefaultSumGeo<S, MP>;

    static S *region(const Problem &p, void *ws, int r) {
        return reinterpret_cast<S *>(static_cast<char *>(ws) + ws_offset(p, sizeof(S), r));
    }

    static unsigned *counters(const Problem &p, void *ws) {
        return reinterpret_cast<unsigned *>(static_cast<char *>(ws) + ws_offset(p, sizeof(S), 7));
    }

    // stages of the first kind in a pass: as many as keep about kL2Keep bytes
    // of `a` in L2 for the next pass
    static int l2_keep(const Problem &p) {
        const int nblk = p.L / SRS < 255 ? p.L / SRS : 255;
        const double rows = p.off != nullptr ? (double)p.T : (double)p.B * (double)p.T;
        const double bytes = rows * (double)p.M * sizeof(S);
        if (bytes <= (double)kL2Keep) return nblk;
        const int k = (int)((double)nblk * (double)kL2Keep / bytes);
        return k < 0 ? 0 : k;
    }

    template <typename G1, bool BWD, int SRC>
    static cudaError_t summary_as(const Problem &p, const Batch &bt, const S *a, const S *u, S *Y, unsigned *cnt,
                                  cudaStream_t st, const CoefSrc &cs) {
        static std::atomic<bool> done[kMaxDevices] = {};
        const int W = k1_warps_for<G1>();
        const size_t smem = (size_t)W * G1::WARP_BYTES;
        auto kern = k1_summary<S, MP, G1::G, G1::R, BWD, SRC>;
        cudaError_t err = allow_smem(kern, smem, done);
        if (err != cudaSuccess) return err;
        const int64_t per_block = (int64_t)W * G1::CPW;
        const int64_t grid = (p.NQ + per_block - 1) / per_block;
        // the next pass (re-run or adjoint re-run) starts on this pass's first stages
        const int l2 = SRC == SRC_STREAM ? l2_word(l2_keep(p), L2_LAST, L2_FIRST) : 0;
        return launch(kern, dim3((unsigned)grid), dim3(32 * W), smem, st, false, bt, p.M, p.L, p.NQ, a, u, Y,
                      p.M == MP ? 1 : 0, cnt, p.B + 1, l2, p.status, cs);
    }

    template <bool BWD, int SRC = SRC_STREAM>
    static cudaError_t summary(const Problem &p, const Batch &bt, const S *a, const S *u, S *Y, unsigned *cnt,
                               cudaStream_t st, const CoefSrc &cs = CoefSrc()) {
        if constexpr (SRC == SRC_STREAM && sizeof(S) == 4) {
            // the autotuner's alternative: twice the lanes per chunk
            if (launch_shape().k1_lane_factor == 2)
                return summary_as<WideSumGeo<S, MP>, BWD, SRC>(p, bt, a, u, Y, cnt, st, cs);
        }
        return summary_as<GE, BWD, SRC>(p, bt, a, u, Y, cnt, st, cs);
    }

    // Two-level scan in one cooperative launch: as many blocks as the items
    // need, at most as many as fit on the device at once.
    static int *fix_list(const Problem &p, void *ws) {
        return reinterpret_cast<int *>(static_cast<char *>(ws) + ws_offset(p, sizeof(S), 9));
    }

    template <int MODE>
    static cudaError_t scan(const Problem &p, const Batch &bt, const S *Y, const S *Z, S *GY, S *GZ, S *GX,
                            const S *zi, S *X, S *ckpt, unsigned *cnt, cudaStream_t st, int *list = nullptr) {
        static std::atomic<bool> done[kMaxDevices] = {};
        static std::atomic<int> resident[kMaxDevices] = {};
        using SG = ScanGeo<S, MP>;
        auto kern = k2_scan<S, MP, MODE>;
        const size_t smem = (size_t)kScanWarps * SG::WARP_BYTES;
        cudaError_t err = allow_smem(kern, smem, done);
        if (err != cudaSuccess) return err;
        int dev = 0;
        if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
        int res = resident[dev].load(std::memory_order_relaxed);
        if (res == 0) {
            int per_sm = 0, sms = 0;
            if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kScanWarps * 32, smem)) !=
                cudaSuccess)
                return err;
            if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            res = per_sm * sms;
            resident[dev].store(res, std::memory_order_relaxed);
        }
        const int64_t items = p.items;
        int64_t blocks = (items + kScanWarps - 1) / kScanWarps;
        // a chain block per signal (phase B1 with the signal's group maps all
        // in its shared memory) when they fit beside one warp per item;
        // otherwise the warp of each signal's first group runs its chain
        const int64_t n_chain = blocks + p.B <= res ? p.B : 0;
        const int chain_regs = ChainRegs<S, MP>::ON ? 1 : 0;
        if (blocks > res) blocks = res;
        return launch(kern, dim3((unsigned)(blocks + n_chain)), dim3(kScanWarps * 32), smem, st, true, bt, p.M, items,
                      Y, Z, GY, GZ, GX, zi, X, ckpt, cnt, p.status, list, (int)n_chain, chain_regs);
    }

    template <int MODE, bool EXACT, int SRC, int RC>
    static cudaError_t rec_as(const Problem &p, const Batch &bt, const S *a, const S *u, const S *Xin, const S *zi,
                              S *out, S *Zout, S *gzi, int reverse, unsigned *cnt, int l2, int xs, cudaStream_t st,
                              const CoefSrc &cs, const S *sfw, S *ga, const Fix<S> &fx) {
        static std::atomic<bool> done[kMaxDevices] = {};
        using RG = RecGeo<S, MP, RC>;
        auto kern = k_rec<S, MP, EXACT, MODE, SRC, RC>;
        constexpr size_t smem = MODE == BWD_GRAD ? RG::SMEM_GA : RG::SMEM;
        cudaError_t err = allow_smem(kern, smem, done);
        if (err != cudaSuccess) return err;
        const int64_t grid = (p.NQ + RC - 1) / RC;
        return launch(kern, dim3((unsigned)grid), dim3(32), smem, st, false, bt, p.M, p.L, p.NQ, a, u, Xin, zi,
                      out, Zout, gzi, reverse, cnt, p.B + 1, l2, xs, p.status, cs, sfw, ga, fx);
    }

    template <int MODE, bool EXACT, int SRC = SRC_STREAM>
    static cudaError_t rec_exact(const Problem &p, const Batch &bt, const S *a, const S *u, const S *Xin,
                                 const S *zi, S *out, S *Zout, S *gzi, int reverse, unsigned *cnt, int l2, int xs,
                                 cudaStream_t st, const CoefSrc &cs = CoefSrc(), const S *sfw = nullptr,
                                 S *ga = nullptr, const Fix<S> &fx = Fix<S>()) {
        if constexpr (SRC == SRC_STREAM && sizeof(S) == 4 && MODE != BWD_GRAD) {
            // the autotuner's alternative: 8 chunks per warp
            if (launch_shape().rec_chunks == 8)
                return rec_as<MODE, EXACT, SRC, 8>(p, bt, a, u, Xin, zi, out, Zout, gzi, reverse, cnt, l2, xs, st, cs,
                                                   sfw, ga, fx);
        }
        return rec_as<MODE, EXACT, SRC, RecChunks<SRC>::N>(p, bt, a, u, Xin, zi, out, Zout, gzi, reverse, cnt, l2, xs,
                                                            st, cs, sfw, ga, fx);
    }

    // one recursion per chunk; `cnt`, when given, is zeroed for a scan that
    // follows; `l2` is the pass's L2 residency word (l2_word)
    template <int MODE>
    static cudaError_t rec(const Problem &p, const Batch &bt, const S *a, const S *u, const S *Xin, const S *zi,
                           S *out, S *Zout, S *gzi, int reverse, cudaStream_t st, unsigned *cnt = nullptr, int l2 = 0,
                           int xs = MP, const Fix<S> &fx = Fix<S>()) {
        if (p.M == MP)
            return rec_exact<MODE, true>(p, bt, a, u, Xin, zi, out, Zout, gzi, reverse, cnt, l2, xs, st, CoefSrc(),
                                         nullptr, nullptr, fx);
        return rec_exact<MODE, false>(p, bt, a, u, Xin, zi, out, Zout, gzi, reverse, cnt, l2, xs, st, CoefSrc(),
                                      nullptr, nullptr, fx);
    }

    // the adjoint re-run that also writes Eq. 12's ga (M == MP only)
    static cudaError_t rec_grad(const Problem &p, const Batch &bt, const S *a, const S *gs, const S *Win, const S *zi,
                                const S *s, S *ge, S *ga, S *gzi, cudaStream_t st, int l2,
                                const Fix<S> &fx = Fix<S>()) {
        return rec_exact<BWD_GRAD, true>(p, bt, a, gs, Win, zi, ge, nullptr, gzi, 1, nullptr, l2, MP, st, CoefSrc(), s,
                                         ga, fx);
    }

    // the same with generated coefficient rows (rows are written whole, so
    // the exact-order kernel serves every M)
    template <int MODE, int SRC>
    static cudaError_t rec_gen(const Problem &p, const Batch &bt, const S *u, const S *Xin, const S *zi, S *out,
                               S *Zout, S *gzi, int reverse, cudaStream_t st, const CoefSrc &cs,
                               unsigned *cnt = nullptr, const Fix<S> &fx = Fix<S>()) {
        return rec_exact<MODE, true, SRC>(p, bt, nullptr, u, Xin, zi, out, Zout, gzi, reverse, cnt, 0, MP, st, cs,
                                          nullptr, nullptr, fx);
    }

    static cudaError_t grad_a(const Problem &p, const Batch &bt, const S *ge, const S *s, const S *zi, S *ga,
                              cudaStream_t st) {
        if ((int64_t)p.B * p.T * p.M == 0) return cudaSuccess;
        constexpr int TR = GradGeo<S, MP, true>::TR;
        // uniform: tiles of TR rows per signal; varlen: tiles of TR packed rows
        const int64_t tiles = (p.T + TR - 1) / TR;
        const int64_t grid = p.off != nullptr ? tiles : tiles * p.B;
        if (p.M == MP)
            return launch(k_grad_a<S, MP, true>, dim3((unsigned)grid), dim3(GradGeo<S, MP, true>::THREADS), 0, st, false,
                          bt, p.M, tiles, ge, s, zi, ga);
        return launch(k_grad_a<S, MP, false>, dim3((unsigned)grid), dim3(GradGeo<S, MP, false>::THREADS), 0, st, false,
                      bt, p.M, tiles, ge, s, zi, ga);
    }
};

// The plain path runs the one-recursion kernels with one chunk per signal.
inline Problem plain_problem(const Problem &p) {
    Problem q = p;
    q.L = (int)(((p.T + SRS - 1) / SRS) * SRS);
    if (q.L == 0) q.L = SRS;
    q.nC = 1;
    q.NQ = p.B;
    return q;
}

// Launch helper: wraps one kernel launch in the profiling marks.
#define TVLP_LAUNCH(K, CALL)                          \
    do {                                              \
        const int k_ = (K);                           \
        profile_mark(k_, false, st);                  \
        if ((CALL) != cudaSuccess) return ECUDA;      \
        profile_mark(k_, true, st);                   \
    } while (0)

// Varlen batches: the per-signal chunk and group tables, rebuilt at the
// start of every call (a plain launch, so the tables are complete before the
// next kernel starts).
inline cudaError_t build_tables(const Problem &p, const Batch &bt, cudaStream_t st) {
    if (p.off == nullptr) return cudaSuccess;
    k_varlen_tables<<<1, kTableThreads, 0, st>>>(p.off, p.B, p.L, const_cast<int *>(bt.cstart),
                                                 const_cast<int *>(bt.gstart));
    return cudaGetLastError();
}

// Defect correction of the chunked scan (see Fix in the kernels): FP32
// calls whose signals have chunk boundaries.  Pass 1 writes the defects
// into the adjoint zero-state region Z (free in a forward, consumed by the
// adjoint's main scan before its pass 1) and each signal's output scale
// into its counter line; the correction scan writes the corrections into a
// state region the call no longer needs (forward: the adjoint's W;
// adjoint: the forward's X).
template <typename S> inline bool refines(const Problem &p) {
    return sizeof(S) == 4 && p.NQ > 0 && (p.off != nullptr || p.nC > 1);
}
template <typename S> inline Fix<S> fix_pass1(S *D, unsigned *cnt) {
    Fix<S> f;
    f.D = D;
    f.scale = cnt;
    return f;
}
template <typename S> inline Fix<S> fix_pass2(const Problem &p, const S *E, unsigned *cnt, const int *list,
                                              S *ckpt = nullptr) {
    Fix<S> f;
    f.E = E;
    f.scale = cnt;
    f.ckpt = ckpt;
    f.list = list;
    f.list_n = cnt + (size_t)p.B * kCntStride;
    return f;
}

template <typename S, int MP>
int Impl<S, MP>::forward(const Problem &p, const S *a, const S *e, const S *zi, S *s, S *ckpt, int algo,
                         void *ws, cudaStream_t st) {
    using LN = Launch<S, MP>;
    if (algo == ALGO_PLAIN) {
        const Problem q = plain_problem(p);
        TVLP_LAUNCH(0, (LN::template rec<FWD_RERUN>(q, batch_of(q, nullptr, sizeof(S)), a, e, nullptr, zi, s,
                                                    nullptr, nullptr, 0, st)));
        return OK;
    }
    const Batch bt = batch_of(p, ws, sizeof(S));
    if (build_tables(p, bt, st) != cudaSuccess) return ECUDA;
    S *Y = LN::region(p, ws, 0);
    S *X = LN::region(p, ws, 1);
    S *GY = LN::region(p, ws, 4);
    S *GX = LN::region(p, ws, 6);
    unsigned *cnt = LN::counters(p, ws);
    TVLP_LAUNCH(0, (LN::template summary<false>(p, bt, a, e, Y, cnt, st)));
    TVLP_LAUNCH(1, (LN::template scan<CH_FWD>(p, bt, Y, nullptr, GY, nullptr, GX, zi, X, ckpt, cnt, st)));
    // the re-run reads the stages K1 kept first, streams the middle and
    // keeps its last stages for an adjoint pass, which walks the chunks the
    // other way
    const int keep = LN::l2_keep(p), nblk = p.L / SRS;
    const bool fix = refines<S>(p);
    S *D = LN::region(p, ws, 2), *E = LN::region(p, ws, 3);
    TVLP_LAUNCH(2, (LN::template rec<FWD_RERUN>(p, bt, a, e, X, zi, s, nullptr, nullptr, 1, st, nullptr,
                                                l2_word(keep, L2_FIRST, L2_FIRST, nblk - keep, L2_LAST), MP,
                                                fix ? fix_pass1<S>(D, cnt) : Fix<S>())));
    if (fix) {
        int *list = LN::fix_list(p, ws);
        TVLP_LAUNCH(3, (LN::template scan<CH_FWD_FIX>(p, bt, Y, D, GY, LN::region(p, ws, 5), GX, nullptr, E, nullptr,
                                                      cnt, st, list)));
        TVLP_LAUNCH(4, (LN::template rec<FWD_RERUN>(p, bt, a, e, X, zi, s, nullptr, nullptr, 1, st, nullptr, 0, MP,
                                                    fix_pass2<S>(p, E, cnt, list, ckpt))));
    }
    return OK;
}

template <typename S, int MP>
int Impl<S, MP>::rerun(const Problem &p, const S *a, const S *e, const S *ckpt, const S *zi, S *s, void *ws,
                       cudaStream_t st) {
    using LN = Launch<S, MP>;
    const Batch bt = batch_of(p, ws, sizeof(S));
    if (build_tables(p, bt, st) != cudaSuccess) return ECUDA;
    // the forward's re-run pass from its stored chunk states: the same kernel
    // on the same states, so s comes out bit for bit as the forward wrote it
    TVLP_LAUNCH(0, (LN::template rec<FWD_RERUN>(p, bt, a, e, ckpt, zi, s, nullptr, nullptr, 1, st, nullptr, 0, p.M)));
    return OK;
}

template <typename S, int MP>
int Impl<S, MP>::backward(const Problem &p, const S *gs, const S *a, const S *s, const S *zi, S *ge, S *ga,
                          S *gzi, int algo, int flags, void *ws, cudaStream_t st) {
    using LN = Launch<S, MP>;
    int k = 0;
    const Problem q = algo == ALGO_PLAIN ? plain_problem(p) : p;
    const Batch bt = batch_of(q, algo == ALGO_PLAIN ? nullptr : ws, sizeof(S));
    // on request (chunked, exact rows): Eq. 12 inside the adjoint re-run;
    // otherwise a separate pass over ge and s
    const bool fused_ga = ga != nullptr && algo != ALGO_PLAIN && p.M == MP && (flags & BWD_FUSED_GA);
    if (algo == ALGO_PLAIN) {
        TVLP_LAUNCH(k++, (LN::template rec<BWD_RERUN>(q, bt, a, gs, nullptr, nullptr, ge, nullptr, gzi, 0, st)));
    } else {
        if (build_tables(p, bt, st) != cudaSuccess) return ECUDA;
        S *Y = LN::region(p, ws, 0);
        S *Z = LN::region(p, ws, 2);
        S *Wst = LN::region(p, ws, 3);
        S *GY = LN::region(p, ws, 4);
        S *GZ = LN::region(p, ws, 5);
        S *GX = LN::region(p, ws, 6);
        unsigned *cnt = LN::counters(p, ws);
        if (flags & BWD_REUSE_FORWARD) {
            // forward transfers P_c (and their group compositions) are in the
            // workspace: the adjoint needs one zero-state recursion per chunk,
            // then w_{c-1} = P_c^T w_c + z_c
            TVLP_LAUNCH(k++, (LN::template rec<BWD_ZERO>(p, bt, a, gs, nullptr, nullptr, nullptr, Z, nullptr, 0, st,
                                                         cnt, l2_word(LN::l2_keep(p), L2_LAST, L2_FIRST))));
            TVLP_LAUNCH(k++,
                        (LN::template scan<CH_TRANS>(p, bt, Y, Z, GY, GZ, GX, nullptr, Wst, nullptr, cnt, st)));
        } else {
            TVLP_LAUNCH(k++, (LN::template summary<true>(p, bt, a, gs, Y, cnt, st)));
            TVLP_LAUNCH(k++,
                        (LN::template scan<CH_BWD>(p, bt, Y, nullptr, GY, nullptr, GX, nullptr, Wst, nullptr, cnt, st)));
        }
        const bool fix = refines<S>(p);
        S *E = LN::region(p, ws, 1);
        auto rerun = [&](const Fix<S> &fx, int l2) -> cudaError_t {
            // with fused_ga the re-run writes ga as it goes (Eq. 12 from its own ge)
            if (fused_ga) return LN::rec_grad(p, bt, a, gs, Wst, zi, s, ge, ga, gzi, st, l2, fx);
            return LN::template rec<BWD_RERUN>(p, bt, a, gs, Wst, nullptr, ge, nullptr, gzi, 1, st, nullptr, l2, MP,
                                               fx);
        };
        TVLP_LAUNCH(k++, (rerun(fix ? fix_pass1<S>(Z, cnt) : Fix<S>(), l2_word(0, L2_FIRST, L2_FIRST))));
        if (fix) {
            int *list = LN::fix_list(p, ws);
            if (flags & BWD_REUSE_FORWARD)
                TVLP_LAUNCH(k++, (LN::template scan<CH_TRANS_FIX>(p, bt, Y, Z, GY, GZ, GX, nullptr, E, nullptr, cnt,
                                                                  st, list)));
            else
                TVLP_LAUNCH(k++, (LN::template scan<CH_BWD_FIX>(p, bt, Y, Z, GY, GZ, GX, nullptr, E, nullptr, cnt,
                                                                st, list)));
            TVLP_LAUNCH(k++, (rerun(fix_pass2<S>(p, E, cnt, list), 0)));
        }
    }
    if (ga != nullptr && !fused_ga) TVLP_LAUNCH(k, (LN::grad_a(q, bt, ge, s, zi, ga, st)));
    return OK;
}

// Forward and adjoint with generated coefficient rows: the chunked path of
// forward / backward with every pass over `a` taking its rows from the
// source (SRC_CONST or SRC_FRAMES).  FP32 only.
template <typename S, int MP, int SRC>
int forward_gen_src(const Problem &p, const CoefSrc &src, const S *e, const S *zi, S *s, S *ckpt, void *ws,
                    cudaStream_t st) {
    using LN = Launch<S, MP>;
    const Batch bt = batch_of(p, ws, sizeof(S));
    if (build_tables(p, bt, st) != cudaSuccess) return ECUDA;
    S *Y = LN::region(p, ws, 0);
    S *X = LN::region(p, ws, 1);
    S *GY = LN::region(p, ws, 4);
    S *GX = LN::region(p, ws, 6);
    unsigned *cnt = LN::counters(p, ws);
    TVLP_LAUNCH(0, (LN::template summary<false, SRC>(p, bt, nullptr, e, Y, cnt, st, src)));
    TVLP_LAUNCH(1, (LN::template scan<CH_FWD>(p, bt, Y, nullptr, GY, nullptr, GX, zi, X, ckpt, cnt, st)));
    auto rerun = [&](const Fix<S> &fx, bool first) -> cudaError_t {
        if (src.cache != nullptr) {
            // the summary pass left every generated row in the cache: stream it
            const int keep = LN::l2_keep(p), nblk = p.L / SRS;
            return LN::template rec_exact<FWD_RERUN, true>(
                p, bt, src.cache, e, X, zi, s, nullptr, nullptr, 1, nullptr,
                first ? l2_word(keep, L2_FIRST, L2_FIRST, nblk - keep, L2_LAST) : 0, MP, st, CoefSrc(), nullptr,
                nullptr, fx);
        }
        return LN::template rec_gen<FWD_RERUN, SRC>(p, bt, e, X, zi, s, nullptr, nullptr, 1, st, src, nullptr, fx);
    };
    const bool fix = refines<S>(p);
    S *D = LN::region(p, ws, 2), *E = LN::region(p, ws, 3);
    TVLP_LAUNCH(2, (rerun(fix ? fix_pass1<S>(D, cnt) : Fix<S>(), true)));
    if (fix) {
        int *list = LN::fix_list(p, ws);
        TVLP_LAUNCH(3, (LN::template scan<CH_FWD_FIX>(p, bt, Y, D, GY, LN::region(p, ws, 5), GX, nullptr, E, nullptr,
                                                      cnt, st, list)));
        TVLP_LAUNCH(4, (rerun(fix_pass2<S>(p, E, cnt, list, ckpt), false)));
    }
    return OK;
}

template <typename S, int MP, int SRC>
int backward_gen_src(const Problem &p, const CoefSrc &src, const S *gs, const S *zi, S *ge, S *gzi, int flags,
                     void *ws, cudaStream_t st) {
    using LN = Launch<S, MP>;
    int k = 0;
    const Batch bt = batch_of(p, ws, sizeof(S));
    if (build_tables(p, bt, st) != cudaSuccess) return ECUDA;
    S *Y = LN::region(p, ws, 0);
    S *Z = LN::region(p, ws, 2);
    S *Wst = LN::region(p, ws, 3);
    S *GY = LN::region(p, ws, 4);
    S *GZ = LN::region(p, ws, 5);
    S *GX = LN::region(p, ws, 6);
    unsigned *cnt = LN::counters(p, ws);
    (void)zi;
    // the forward's cached rows (valid with its workspace only)
    const S *rows = (flags & BWD_REUSE_FORWARD) ? src.cache : nullptr;
    if (rows != nullptr) {
        TVLP_LAUNCH(k++, (LN::template rec_exact<BWD_ZERO, true>(p, bt, rows, gs, nullptr, nullptr, nullptr, Z, nullptr,
                                                                 0, cnt, l2_word(LN::l2_keep(p), L2_LAST, L2_FIRST),
                                                                 MP, st)));
        TVLP_LAUNCH(k++, (LN::template scan<CH_TRANS>(p, bt, Y, Z, GY, GZ, GX, nullptr, Wst, nullptr, cnt, st)));
    } else if (flags & BWD_REUSE_FORWARD) {
        TVLP_LAUNCH(k++, (LN::template rec_gen<BWD_ZERO, SRC>(p, bt, gs, nullptr, nullptr, nullptr, Z, nullptr, 0, st,
                                                              src, cnt)));
        TVLP_LAUNCH(k++, (LN::template scan<CH_TRANS>(p, bt, Y, Z, GY, GZ, GX, nullptr, Wst, nullptr, cnt, st)));
    } else {
        TVLP_LAUNCH(k++, (LN::template summary<true, SRC>(p, bt, nullptr, gs, Y, cnt, st, src)));
        TVLP_LAUNCH(k++, (LN::template scan<CH_BWD>(p, bt, Y, nullptr, GY, nullptr, GX, nullptr, Wst, nullptr, cnt,
                                                    st)));
    }
    auto rerun = [&](const Fix<S> &fx, int l2) -> cudaError_t {
        if (rows != nullptr)
            return LN::template rec_exact<BWD_RERUN, true>(p, bt, rows, gs, Wst, nullptr, ge, nullptr, gzi, 1, nullptr,
                                                           l2, MP, st, CoefSrc(), nullptr, nullptr, fx);
        return LN::template rec_gen<BWD_RERUN, SRC>(p, bt, gs, Wst, nullptr, ge, nullptr, gzi, 1, st, src, nullptr,
                                                     fx);
    };
    const bool fix = refines<S>(p);
    S *E = LN::region(p, ws, 1);
    TVLP_LAUNCH(k++, (rerun(fix ? fix_pass1<S>(Z, cnt) : Fix<S>(), l2_word(0, L2_FIRST, L2_FIRST))));
    if (fix) {
        int *list = LN::fix_list(p, ws);
        if (flags & BWD_REUSE_FORWARD)
            TVLP_LAUNCH(k++,
                        (LN::template scan<CH_TRANS_FIX>(p, bt, Y, Z, GY, GZ, GX, nullptr, E, nullptr, cnt, st, list)));
        else
            TVLP_LAUNCH(k++,
                        (LN::template scan<CH_BWD_FIX>(p, bt, Y, Z, GY, GZ, GX, nullptr, E, nullptr, cnt, st, list)));
        TVLP_LAUNCH(k++, (rerun(fix_pass2<S>(p, E, cnt, list), 0)));
    }
    return OK;
}

template <typename S, int MP>
int Impl<S, MP>::forward_gen(const Problem &p, const CoefSrc &src, const S *e, const S *zi, S *s, S *ckpt, void *ws,
                             cudaStream_t st) {
    if constexpr (sizeof(S) != 4) {
        return EUNSUPPORTED;
    } else {
        if (src.kind == SRC_CONST) return forward_gen_src<S, MP, SRC_CONST>(p, src, e, zi, s, ckpt, ws, st);
        if (src.kind == SRC_FRAMES) return forward_gen_src<S, MP, SRC_FRAMES>(p, src, e, zi, s, ckpt, ws, st);
        return EINVAL_;
    }
}

template <typename S, int MP>
int Impl<S, MP>::backward_gen(const Problem &p, const CoefSrc &src, const S *gs, const S *s, const S *zi, S *ge,
                              S *gzi, int flags, void *ws, cudaStream_t st) {
    (void)s;
    if constexpr (sizeof(S) != 4) {
        return EUNSUPPORTED;
    } else {
        if (src.kind == SRC_CONST) return backward_gen_src<S, MP, SRC_CONST>(p, src, gs, zi, ge, gzi, flags, ws, st);
        if (src.kind == SRC_FRAMES)
            return backward_gen_src<S, MP, SRC_FRAMES>(p, src, gs, zi, ge, gzi, flags, ws, st);
        return EINVAL_;
    }
}

template <typename S, int MP>
int Impl<S, MP>::grad_src(const Problem &p, const CoefSrc &src, const S *ge, const S *s, const S *zi, S *gk,
                          void *scratch, cudaStream_t st) {
    if constexpr (sizeof(S) != 4) {
        return EUNSUPPORTED;
    } else {
        float *sc = static_cast<float *>(scratch);
        if (src.kind == SRC_CONST) {
            if (p.off != nullptr) return EUNSUPPORTED;
            const int64_t tiles = (p.T + kGradRows - 1) / kGradRows;
            // profiling slots 5 and 6: after the adjoint's kernels (three,
            // and the two of the defect correction)
            TVLP_LAUNCH(5, (launch(k_grad_const<MP>, dim3((unsigned)tiles, (unsigned)p.B), dim3(kGradThreads), 0, st,
                                   false, p.T, p.M, tiles, ge, s, zi, sc)));
            const int64_t n = (int64_t)p.B * p.M;
            TVLP_LAUNCH(6, (launch(k_grad_const_finish, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, false, p.B,
                                   p.M, MP, tiles, sc, gk)));
            return OK;
        }
        if (src.kind == SRC_FRAMES) {
            using FG = FrameGradGeo<MP>;
            // varlen: src.F is the total number of packed frame rows
            const int64_t items = p.off != nullptr ? src.F : (int64_t)p.B * src.F;
            const int64_t n = items * p.M;
            float *lo = sc, *hi = sc + n;
            TVLP_LAUNCH(5, (launch(k_grad_frames<MP>, dim3((unsigned)((items + FG::WARPS - 1) / FG::WARPS)),
                                   dim3(32 * FG::WARPS), 0, st, false, p.B, p.T, p.M, src.F, src.hop, src.inv_hop,
                                   src.k, ge, s, zi, lo, hi, p.off, src.foff)));
            TVLP_LAUNCH(6, (launch(k_grad_frames_finish, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, false, n,
                                   lo, hi, gk)));
            return OK;
        }
        return EINVAL_;
    }
}

#undef TVLP_LAUNCH

}  // namespace tvlp
