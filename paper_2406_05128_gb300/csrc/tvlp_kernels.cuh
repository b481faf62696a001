// Device kernels of the time-varying LP library (sm_103a).
//
// The filter (Eq. 5 of Yu & Fazekas, arXiv 2406.05128)
//     s(t) = e(t) - sum_{i=1..M} a_i(t) s(t-i)
// is a linear recurrence on the state x_t = [s(t-1), ..., s(t-M)]:
//     x_{t+1} = C(t) x_t + e(t) u_1,   C(t) the companion matrix of a(t).
// Its adjoint (Eq. 11) runs the same filter backwards in time with the
// lag-shifted coefficients a^_i(t) = a_i(t+i).  Here the adjoint is evaluated
// in the transposed ("scatter") form
//     ge(t) = gs(t) + q_1,  q_k <- q_{k+1} - a_k(t) ge(t),  q_M <- -a_M(t) ge(t)
// where, after processing every step >= t, q_k is the pending contribution to
// dL/de(t-k) -- which equals dL/ds(t-k) through all later steps, i.e. the
// gradient with respect to the forward state x_t.  Expanding the pending sums
// gives exactly ge(t) = gs(t) - sum_i a_i(t+i) ge(t+i) (Eq. 11), but this form
// reads only row a(t) at step t.  Because q is the state gradient, the
// adjoint's transfer over a chunk is the transpose of the forward's.  After
// the last step (t = 0), q_j = dL/ds(-j), the initial-state gradient.
//
// Parallel scan over time.  A signal is cut into chunks of L samples (L a
// multiple of SRS = 16), streamed in stages of SRS rows and computed in
// blocks of SR = 8 rows.
//   k1_summary      per chunk, the end states of MP+1 recursions: zero state
//                   driven by the input (column 0) and the MP unit initial
//                   states with zero input (columns 1..MP, the chunk transfer
//                   P_c).  Forward direction; also available backwards.
//   k_rec (ZERO)    per chunk, one recursion from zero state; end state only
//                   (the adjoint's zero-state summary z_c).
//   k2_scan         x_{c+1} = P_c x_c + y_c (forward) or
//                   w_{c-1} = P_c^T w_c + z_c (adjoint) per signal, as a
//                   two-level scan over groups of chunks in one launch.
//   k_rec (RERUN)   each chunk re-runs its recursion from its true incoming
//                   state and writes s (forward) or ge (adjoint).  With one
//                   chunk per signal this is the plain sequential filter.
//   k_grad_a        dL/da_i(t) = -ge(t) s(t-i) (Eq. 12), tiled.
// Orders are padded to MP (compile time); coefficients of order > M are
// zero, which leaves every result unchanged.  Rows past the end of a signal
// are staged as zeros: in the forward they follow its last output, in the
// adjoint they precede its first step with a zero pending state, so both
// leave every result unchanged.
//
// Register state.  A recursion keeps a window of MP + SR values: the MP
// values entering a stage, then the SR values the stage produces.  Every
// index is a compile-time constant inside the unrolled stage; at the end of
// the stage the window slides down by SR (MP moves).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tvlp_impl.h"

namespace tvlp {

constexpr int SR = 8;    // rows per compute block (register window)
constexpr int SRS = 16;  // rows per staged copy; chunk lengths are multiples of SRS

// Status codes written by kernels to the device status word.
enum { DEV_OK = 0, DEV_TIMEOUT_TMA = 1, DEV_TIMEOUT_SCAN = 2 };

// Index checks of a checked build (TVLP_CHECK_BOUNDS): the indices that come
// from tables and lists built on the device are checked against the ranges
// they must lie in.  A failed check records DEV_BOUNDS + its location in
// the status word (the first failure wins) and the caller skips the work
// the index guards; nothing traps.  Other builds compile the checks out.
constexpr int DEV_BOUNDS = 16;
enum {
    CHK_FIX_LIST_ENTRY = 1,  // pass 2: a listed chunk outside [0, NQ)
    CHK_CHUNK_SIGNAL = 2,    // a varlen chunk outside its signal's chunks
    CHK_SCAN_ITEM = 3,       // a scan item outside its signal's groups
    CHK_SCAN_CHUNK = 4,      // a group's chunks outside the batch's chunks
    CHK_FIX_LIST_SLOT = 5,   // the correction list past the batch's chunks
    CHK_CHAIN_GROUPS = 6,    // a chain's groups past the scan items
};
#ifdef TVLP_CHECK_BOUNDS
__device__ __forceinline__ bool index_ok(bool ok, int where, int *status) {
    if (!ok) atomicCAS(status, 0, DEV_BOUNDS + where);
    return ok;
}
#else
__device__ __forceinline__ bool index_ok(bool, int, int *) { return true; }
#endif

constexpr int kCntStride = 32;  // scan counters sit 128 bytes apart, one L2 line each

// Packing of the MP+1 summary recursions of one chunk onto G lanes with R
// recursions per lane (G*R >= MP+1).  A warp holds 32/G chunks.
template <int MP> struct Pack;
template <> struct Pack<2>  { static constexpr int G = 1,  R = 3; };
template <> struct Pack<4>  { static constexpr int G = 1,  R = 5; };
template <> struct Pack<8>  { static constexpr int G = 2,  R = 5; };
template <> struct Pack<12> { static constexpr int G = 2,  R = 7; };
template <> struct Pack<16> { static constexpr int G = 4,  R = 5; };
template <> struct Pack<22> { static constexpr int G = 4,  R = 6; };
template <> struct Pack<30> { static constexpr int G = 8,  R = 4; };
template <> struct Pack<32> { static constexpr int G = 16, R = 3; };
// The alternative packing the autotuner can choose: twice the lanes per
// chunk, half the recursions per lane (more threads per signal, fewer
// independent chains per lane; odd R runs without packed pairs).
template <int MP> struct PackWide;
template <> struct PackWide<2>  { static constexpr int G = 2,  R = 2; };
template <> struct PackWide<4>  { static constexpr int G = 2,  R = 3; };
template <> struct PackWide<8>  { static constexpr int G = 4,  R = 3; };
template <> struct PackWide<12> { static constexpr int G = 4,  R = 4; };
template <> struct PackWide<16> { static constexpr int G = 8,  R = 3; };
template <> struct PackWide<22> { static constexpr int G = 8,  R = 3; };
template <> struct PackWide<30> { static constexpr int G = 16, R = 2; };
template <> struct PackWide<32> { static constexpr int G = 32, R = 2; };

// Bank-conflict helper: `groups` readers at multiples of `stride_words`
// reading 8-byte words; worst number of readers sharing a bank pair.
constexpr int pair_conflicts(int stride_words, int groups) {
    int worst = 1;
    for (int x = 0; x < groups; ++x) {
        int n = 0;
        for (int y = 0; y < groups; ++y)
            if (((x * stride_words) / 2) % 16 == ((y * stride_words) / 2) % 16) ++n;
        worst = n > worst ? n : worst;
    }
    return worst;
}
// padding (a multiple of `step` words, below 32) with the fewest conflicts
constexpr int conflict_free_pad(int base_words, int groups, int step) {
    int best = 0, best_n = pair_conflicts(base_words, groups);
    for (int p = step; p < 32; p += step) {
        const int n = pair_conflicts(base_words + p, groups);
        if (n < best_n) {
            best = p;
            best_n = n;
        }
    }
    return best;
}
__host__ __device__ constexpr int wrapm(int x, int m) { return ((x % m) + m) % m; }

// Geometry of the summary kernel for packing (G, R).
template <typename S, int MP, int G_, int R_> struct SumGeo {
    static constexpr int G = G_, R = R_;
    static constexpr int CPW = 32 / G;                     // chunks per warp
    static constexpr int NS = 2;                            // stages in the ring
    static constexpr int WPS = (int)sizeof(S) / 4;          // 32-bit words per element
    static constexpr int GPH = (16 / G) > 1 ? 16 / G : 1;   // chunk groups per half-warp
    // chunk-stage stride (elements): SRS rows of MP coefficients + padding,
    // a multiple of 16 bytes (bulk-copy destination)
    static constexpr int CS = SRS * MP + conflict_free_pad(SRS * MP * WPS, GPH, 4) / WPS;
    static constexpr int A_STAGE = CPW * CS;
    static constexpr int U_STAGE = CPW * SRS;               // input samples of a stage
    // per-warp slice: the stage ring then NS mbarriers, rounded to 128 bytes
    // so every warp's bulk-copy destinations stay 16-byte aligned
    static constexpr size_t RING_BYTES = size_t(NS) * (A_STAGE + U_STAGE) * sizeof(S);
    static constexpr size_t WARP_BYTES = ((RING_BYTES + NS * 8 + 127) / 128) * 128;
    static_assert(G * R >= MP + 1, "packing must hold MP+1 recursions");
    static_assert((CS * sizeof(S)) % 16 == 0, "16-byte stage alignment");
    static_assert((A_STAGE * sizeof(S)) % 16 == 0 && (U_STAGE * sizeof(S)) % 16 == 0, "16-byte ring alignment");
    static_assert(RING_BYTES % 8 == 0 && WARP_BYTES % 16 == 0, "mbarrier and warp-slice alignment");
};
// chunk summaries Y[c][MP+1][RS]: rows of MP values padded to RS, a 16-byte
// multiple, so that every row starts 16-byte aligned (vector loads of a row)
template <typename S, int MP> struct YGeo {
    static constexpr int RS = ((MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
    static constexpr int YS = (MP + 1) * RS;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// Asynchronous global->shared copy of BYTES (4, 8 or 16); only the first
// `src_bytes` are read, the rest of the destination is zero-filled.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, int src_bytes) {
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                     "r"(src_bytes)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)), "l"(src),
                     "n"(BYTES), "r"(src_bytes)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// mbarrier + 1-D bulk (TMA) copies
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for an mbarrier phase by every lane of the warp; the outcome
// is warp-uniform (false if any lane gave up after `limit` polls).
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, unsigned parity, int limit) {
    bool ok = false;
    for (int i = 0; i < limit && !ok; ++i) ok = mbar_try_wait(bar, parity);
    return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
// 1-D bulk store shared -> global in the issuing thread's bulk groups
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the thread's stores have finished reading their shared source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// the thread's stores but its newest group have read their shared source
__device__ __forceinline__ void bulk_wait_read_prev() {
    asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
}
// the thread's stores are complete in global memory
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_store_commit_wait() {
    bulk_commit();
    bulk_wait_all();
}

// Programmatic dependent launch.  The kernels of one call run back to back
// on a stream; each may be launched before the previous one has finished.
// pdl_wait() returns once the previous kernel has completed and its writes
// are visible (immediately when launched without the attribute); only after
// it does a kernel touch data the previous kernel writes or reads, and only
// then does it let the next kernel launch (pdl_release), so that work a
// kernel does before its wait overlaps its immediate predecessor alone.
// Before the wait kernels only read the call's inputs (coefficients,
// excitation, upstream gradient, and results of kernels two or more
// launches back).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Packed pairs of floats (two lanes of one register pair) and the packed
// IEEE fma: fma.rn.f32x2 rounds each half exactly like fmaf.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(unsigned long long r) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
    return lo;
}
__device__ __forceinline__ float f2_hi(unsigned long long r) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
    return hi;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// L2 residency of the coefficient stages a pass reads.  Consecutive passes
// over `a` reuse what L2 still holds from the previous one: a pass keeps the
// stages the next pass reads first (evict_last) and streams the rest
// (evict_first); the next pass reads the kept stages evict_first.  A launch
// gets one word: in its own stage order, stages [0, head_n) use policy
// `head`, stages [tail_from, ...) policy `tail`, the others policy `mid`
// (L2_NORMAL: no hint).
enum { L2_NORMAL = 0, L2_FIRST = 1, L2_LAST = 2 };
__host__ __device__ constexpr int l2_word(int head_n, int head, int mid, int tail_from = 0xff, int tail = 0) {
    return (head_n & 0xff) | ((tail_from & 0xff) << 8) | (head << 16) | (mid << 18) | (tail << 20);
}
__device__ __forceinline__ int l2_kind(int word, int stage) {
    if (stage < (word & 0xff)) return (word >> 16) & 3;
    if (stage >= ((word >> 8) & 0xff)) return (word >> 20) & 3;
    return (word >> 18) & 3;
}
__device__ __forceinline__ void bulk_load_l2(void *dst, const void *src, unsigned bytes, uint64_t *bar, int kind) {
    if (kind == L2_NORMAL) {
        bulk_load(dst, src, bytes, bar);
        return;
    }
    uint64_t pol;
    if (kind == L2_LAST) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(pol));
    else asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

// Prefetch [p, p + bytes) into L2 (one bulk prefetch of the 16-byte
// aligned span inside it; nothing outside the range is touched).
__device__ __forceinline__ void l2_prefetch(const void *p, size_t bytes) {
    const uintptr_t lo = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    const uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

constexpr int kWaitLimit = 1 << 18;  // mbarrier polls before a wait gives up (well under a second)

// Load the MP coefficients of one shared-memory row (8-byte aligned for
// float, 16-byte for double; MP is even) into registers.
template <typename S, int MP>
__device__ __forceinline__ void load_row_smem(S (&c)[MP], const S *row) {
    if constexpr (sizeof(S) == 4) {
        const float2 *p = reinterpret_cast<const float2 *>(row);
#pragma unroll
        for (int i = 0; i < MP / 2; ++i) {
            const float2 v = p[i];
            c[2 * i] = v.x;
            c[2 * i + 1] = v.y;
        }
    } else {
        const double2 *p = reinterpret_cast<const double2 *>(row);
#pragma unroll
        for (int i = 0; i < MP / 2; ++i) {
            const double2 v = p[i];
            c[2 * i] = v.x;
            c[2 * i + 1] = v.y;
        }
    }
}
// Load two consecutive rows (16-byte aligned) with 16-byte loads.
template <typename S, int MP>
__device__ __forceinline__ void load_pair_smem(S (&c0)[MP], S (&c1)[MP], const S *rows) {
    S v[2 * MP];
    if constexpr (sizeof(S) == 4) {
        const float4 *p = reinterpret_cast<const float4 *>(rows);
#pragma unroll
        for (int i = 0; i < MP / 2; ++i) {
            const float4 x = p[i];
            v[4 * i] = x.x;
            v[4 * i + 1] = x.y;
            v[4 * i + 2] = x.z;
            v[4 * i + 3] = x.w;
        }
    } else {
        const double2 *p = reinterpret_cast<const double2 *>(rows);
#pragma unroll
        for (int i = 0; i < MP; ++i) {
            const double2 x = p[i];
            v[2 * i] = x.x;
            v[2 * i + 1] = x.y;
        }
    }
#pragma unroll
    for (int i = 0; i < MP; ++i) {
        c0[i] = v[i];
        c1[i] = v[MP + i];
    }
}

// Eq. 12 for two consecutive rows r0, r0 + 1 into shared memory (16-byte
// aligned pair): row r gets -g_r s(t_r - 1 - i), i < MP, where sv[MP + r - 1
// - i] holds s(t_r - 1 - i).
template <typename S, int MP, int NV>
__device__ __forceinline__ void store_ga_pair(S *rows, S g0, S g1, const S (&sv)[NV], int r0) {
    S v[2 * MP];
#pragma unroll
    for (int i = 0; i < MP; ++i) {
        v[i] = -g0 * sv[MP + r0 - 1 - i];
        v[MP + i] = -g1 * sv[MP + r0 - i];
    }
    if constexpr (sizeof(S) == 4) {
        float4 *p = reinterpret_cast<float4 *>(rows);
#pragma unroll
        for (int i = 0; i < MP / 2; ++i) p[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
        double2 *p = reinterpret_cast<double2 *>(rows);
#pragma unroll
        for (int i = 0; i < MP; ++i) p[i] = make_double2(v[2 * i], v[2 * i + 1]);
    }
}

// Forward step on a window h (h[MP + j - i] = s(t - i)); writes s(t) to
// h[MP + j].  Partial sums over the older terms keep the critical path to a
// few FMAs per step.
template <typename S, int MP, int W>
__device__ __forceinline__ S fwd_step_win(S (&h)[W], const S (&c)[MP], S u, int j) {
    S p0 = u, p1 = S(0), p2 = S(0), p3 = S(0);
#pragma unroll
    for (int i = MP; i >= 3; --i) {
        const S hv = h[MP + j - i];
        if ((i & 3) == 0) p0 = fma(-c[i - 1], hv, p0);
        else if ((i & 3) == 1) p1 = fma(-c[i - 1], hv, p1);
        else if ((i & 3) == 2) p2 = fma(-c[i - 1], hv, p2);
        else p3 = fma(-c[i - 1], hv, p3);
    }
    S acc = (p0 + p1) + (p2 + p3);
    if constexpr (MP >= 2) acc = fma(-c[1], h[MP + j - 2], acc);
    acc = fma(-c[0], h[MP + j - 1], acc);
    h[MP + j] = acc;
    return acc;
}

// Adjoint step on a window q: before step j, q_k sits at q[j + k - 1]; after
// it, q_k sits at q[j + k].  Returns ge(t).
template <typename S, int MP, int W>
__device__ __forceinline__ S bwd_step_win(S (&q)[W], const S (&c)[MP], S u, int j) {
    const S y = u + q[j];
#pragma unroll
    for (int k = 1; k < MP; ++k) q[j + k] = fma(-c[k - 1], y, q[j + k]);
    q[j + MP] = -c[MP - 1] * y;
    return y;
}

// slide a window down by SR
template <typename S, int MP, int W>
__device__ __forceinline__ void slide(S (&h)[W]) {
#pragma unroll
    for (int i = 0; i < MP; ++i) h[i] = h[i + SR];
}

// ---------------------------------------------------------------------------
// Where a batch's chunks lie.  Uniform: n signals of T samples, signal b at
// row b*T, nC chunks of L rows each.  Varlen (off != nullptr): signals packed
// back to back, signal b at rows [off[b], off[b+1]); cstart[b] and gstart[b]
// (prefix tables built by k_varlen_tables) number the first chunk and the
// first scan group of signal b, with cstart[n], gstart[n] the totals.  Every
// signal is cut into chunks of L rows from its own start, and its scan groups
// hold group_size(nC_b) chunks, so a signal's results do not depend on the
// rest of the batch.
// ---------------------------------------------------------------------------
struct Batch {
    int64_t T;           // uniform: samples per signal
    int64_t nC;          // uniform: chunks per signal
    int G2, nG;          // uniform: chunks per scan group, groups per signal
    const int64_t *off;  // varlen: [n+1] first row of every signal, or nullptr
    const int *cstart;   // varlen: [n+1] first chunk of every signal
    const int *gstart;   // varlen: [n+1] first scan group of every signal
    int n;               // signals
    // Mixed orders (one class of signals that share a padded order inside a
    // batch of signals of different orders; nullptr otherwise): signal b of
    // the class is signal sig[b] of the batch, with rows
    // [off[sig[b]], off[sig[b]+1]), order ord[sig[b]], coefficient rows of
    // that order starting at element aoff[sig[b]] of a, and initial state
    // at zi[sig[b] * ldz]
    const int *sig;
    const int *ord;
    const int64_t *aoff;
    int ldz;
};

// The batch-wide index of class signal b.
__device__ __forceinline__ int64_t global_signal(const Batch &bt, int64_t b) {
    return bt.sig != nullptr ? (int64_t)__ldg(bt.sig + b) : b;
}

// chunks per scan group for a signal of nC chunks: about sqrt(nC / 4)
__host__ __device__ inline int group_size(int64_t nC) {
    int g = 1;
    while ((int64_t)g * g * 4 < nC) ++g;
    return g;
}

// largest b in [0, n) with start[b] <= x (start non-decreasing, start[0] = 0)
__device__ __forceinline__ int find_signal(const int *__restrict__ start, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)__ldg(start + mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// chunks in the batch (the host sizes grids for an upper bound)
__device__ __forceinline__ int64_t batch_chunks(const Batch &bt, int64_t bound) {
    if (bt.off == nullptr) return bound;
    const int64_t n = __ldg(bt.cstart + bt.n);
    return n < bound ? n : bound;
}

struct ChunkPos {
    int64_t b, c;   // signal (in the class, for mixed orders), chunk within the signal
    int64_t base;   // row of the chunk's first sample
    int valid;      // rows of the chunk inside the signal (<= L)
    int64_t g;      // the signal's index in the batch
    int m;          // its order
    int64_t abase;  // element of `a` where the chunk's coefficient rows start (rows of m)
};
// M: the call's order (every signal's, unless the batch has mixed orders)
__device__ __forceinline__ ChunkPos chunk_pos(const Batch &bt, int64_t q, int L, int M) {
    ChunkPos p;
    int64_t len;
    if (bt.off == nullptr) {
        p.b = q / bt.nC;
        p.c = q - p.b * bt.nC;
        p.base = p.b * bt.T + p.c * (int64_t)L;
        len = bt.T;
        p.g = p.b;
    } else {
        p.b = find_signal(bt.cstart, bt.n, q);
        p.c = q - __ldg(bt.cstart + p.b);
        p.g = global_signal(bt, p.b);
        const int64_t o = __ldg(bt.off + p.g);
        p.base = o + p.c * (int64_t)L;
        len = __ldg(bt.off + p.g + 1) - o;
    }
    if (bt.ord != nullptr) {
        p.m = __ldg(bt.ord + p.g);
        p.abase = __ldg(bt.aoff + p.g) + p.c * (int64_t)L * p.m;
    } else {
        p.m = M;
        p.abase = p.base * (int64_t)M;
    }
    const int64_t rem = len - p.c * (int64_t)L;
    p.valid = rem < 0 ? 0 : (rem < L ? (int)rem : L);
    return p;
}

// ---------------------------------------------------------------------------
// Generated coefficient rows (CoefSrc, FP32).  gen_row writes a(t) of signal
// b, sample t, as MP floats (zero past the order M, or for an invalid row).
//   SRC_CONST:  the signal's one row k[b][0..M).
//   SRC_FRAMES: k(t) = k[f] + w (k[f+1] - k[f]), f = t / hop,
//               w = (t - f hop) / hop (Sec. 4.3: per-sample linear
//               interpolation of the frame-rate reflection coefficients),
//               then the step-up to the direct form of A(z) = 1 + sum a_i z^-i:
//               a^(m)_i = a^(m-1)_i + k_m a^(m-1)_{m-i}, a^(m)_m = k_m.
// ---------------------------------------------------------------------------
template <int MP>
__device__ __forceinline__ void stepup_row(float (&a)[MP], const float *__restrict__ k0,
                                           const float *__restrict__ k1, float w, int M) {
#pragma unroll
    for (int m = 0; m < MP; ++m) a[m] = 0.f;
#pragma unroll
    for (int m = 1; m <= MP; ++m) {
        float km = 0.f;
        if (m <= M) {
            const float x0 = __ldg(k0 + m - 1), x1 = __ldg(k1 + m - 1);
            km = fmaf(w, x1 - x0, x0);
        }
        // pairs (i, m - i) read the old values of both
#pragma unroll
        for (int i = 1; 2 * i < m; ++i) {
            const float lo = a[i - 1], hi = a[m - i - 1];
            a[i - 1] = fmaf(km, hi, lo);
            a[m - i - 1] = fmaf(km, lo, hi);
        }
        if (m % 2 == 0) a[m / 2 - 1] = fmaf(km, a[m / 2 - 1], a[m / 2 - 1]);
        a[m - 1] = km;
    }
}

template <int MP, int SRC>
__device__ __forceinline__ void gen_row(const CoefSrc &cs, int M, int64_t b, int64_t t, bool valid, float *dst) {
    float a[MP];
    if (!valid) {
#pragma unroll
        for (int m = 0; m < MP; ++m) a[m] = 0.f;
    } else if constexpr (SRC == SRC_CONST) {
#pragma unroll
        for (int m = 0; m < MP; ++m) a[m] = m < M ? __ldg(cs.k + b * M + m) : 0.f;
    } else {
        const int64_t f0 = cs.foff != nullptr ? __ldg(cs.foff + b) : b * cs.F;
        // t < 2^31 (the library rejects longer signals): 32-bit division
        const unsigned f = (unsigned)t / (unsigned)cs.hop;
        const float w = (float)((unsigned)t - f * (unsigned)cs.hop) * cs.inv_hop;
        const float *k0 = cs.k + (f0 + (int64_t)f) * (int64_t)M;
        stepup_row<MP>(a, k0, k0 + M, w, M);
    }
    // rows are MP floats (MP even): 8-byte stores
#pragma unroll
    for (int m = 0; m < MP; m += 2) *reinterpret_cast<float2 *>(dst + m) = make_float2(a[m], a[m + 1]);
}

// Two rows per call: two independent step-ups in one basic block, which
// the compiler interleaves (the rows' dependency chains overlap).
template <int MP, int SRC>
__device__ __forceinline__ void gen_rows2(const CoefSrc &cs, int M, int64_t b0, int64_t t0, bool v0, float *d0,
                                          int64_t b1, int64_t t1, bool v1, float *d1) {
    gen_row<MP, SRC>(cs, M, b0, t0, v0, d0);
    gen_row<MP, SRC>(cs, M, b1, t1, v1, d1);
}

// Per-signal scan geometry: first chunk, chunks, first group, groups, group size.
struct SigScan {
    int64_t cbase, nC, gbase;
    int nG, G2;
};
__device__ __forceinline__ SigScan sig_scan(const Batch &bt, int64_t b) {
    SigScan r;
    if (bt.off == nullptr) {
        r.cbase = b * bt.nC;
        r.nC = bt.nC;
        r.gbase = b * bt.nG;
        r.nG = bt.nG;
        r.G2 = bt.G2;
    } else {
        r.cbase = __ldg(bt.cstart + b);
        r.nC = __ldg(bt.cstart + b + 1) - r.cbase;
        r.gbase = __ldg(bt.gstart + b);
        r.nG = (int)(__ldg(bt.gstart + b + 1) - r.gbase);
        r.G2 = group_size(r.nC);
    }
    return r;
}

// Builds the varlen prefix tables: one block; thread i handles a run of
// consecutive signals, then the block scans the runs' totals.
constexpr int kTableThreads = 1024;
static __global__ void __launch_bounds__(kTableThreads)
    k_varlen_tables(const int64_t *__restrict__ off, int n, int L, int *__restrict__ cstart, int *__restrict__ gstart) {
    __shared__ long long sc[kTableThreads], sg[kTableThreads];
    const int t = threadIdx.x;
    const int per = (n + kTableThreads - 1) / kTableThreads;
    const int lo = t * per, hi = (lo + per < n) ? lo + per : n;
    long long nc = 0, ng = 0;
    for (int b = lo; b < hi; ++b) {
        const int64_t len = off[b + 1] - off[b];
        const int64_t c = len > 0 ? (len + L - 1) / L : 0;
        nc += c;
        ng += c > 0 ? (c + group_size(c) - 1) / group_size(c) : 0;
    }
    sc[t] = nc;
    sg[t] = ng;
    __syncthreads();
    for (int d = 1; d < kTableThreads; d <<= 1) {  // inclusive scan
        const long long xc = t >= d ? sc[t - d] : 0, xg = t >= d ? sg[t - d] : 0;
        __syncthreads();
        sc[t] += xc;
        sg[t] += xg;
        __syncthreads();
    }
    long long c0 = sc[t] - nc, g0 = sg[t] - ng;  // exclusive
    for (int b = lo; b < hi; ++b) {
        cstart[b] = (int)c0;
        gstart[b] = (int)g0;
        const int64_t len = off[b + 1] - off[b];
        const int64_t c = len > 0 ? (len + L - 1) / L : 0;
        c0 += c;
        g0 += c > 0 ? (c + group_size(c) - 1) / group_size(c) : 0;
    }
    if (t == kTableThreads - 1) {
        cstart[n] = (int)sc[t];
        gstart[n] = (int)sg[t];
    }
}

// ---------------------------------------------------------------------------
// K1: chunk summaries.
// Flattened chunk index q = b*nC + c; chunk c of signal b covers samples
// [c*L, c*L + L).  Each warp owns CPW consecutive chunks; lane (grp = lane/G,
// g = lane%G) runs recursions r = g*R + k, k < R.  Coefficient rows are
// staged in shared memory, SRS rows per stage, two stages in a ring: a full,
// 16-byte-aligned chunk-stage arrives as one bulk (TMA) copy completing on
// the stage's mbarrier; others (a ragged tail, a misaligned start, a padded
// order) use cp.async with zero fill.  The stage's input samples travel in
// the same cp.async group, into a slot next to the coefficients.
// Output Y[q][r][k] (per-chunk stride YS):
//   forward:  s(c*L + L - 1 - k) of recursion r
//   backward: q_{k+1} after the chunk, i.e. the pending dL/ds(c*L - 1 - k)
// ---------------------------------------------------------------------------
template <typename S, int MP, typename GE, bool BWD>
__device__ __forceinline__ void k1_issue_stage(S *a_st, uint64_t *bar, const S *__restrict__ a, int L, int k,
                                               int lane, int64_t my_abase, int my_m, int my_valid, bool exact,
                                               int l2) {
    constexpr int CPW = GE::CPW;
    constexpr unsigned A_BYTES = SRS * MP * sizeof(S);
    const int roff = BWD ? L - (k + 1) * SRS : k * SRS;  // chunk-local first row of the stage
    int nvalid = my_valid - roff;
    nvalid = nvalid < 0 ? 0 : (nvalid > SRS ? SRS : nvalid);
    const bool mine = lane < CPW;
    const S *src_a = a + my_abase + (int64_t)roff * MP;
    const bool tma_a = mine && exact && nvalid == SRS && aligned16(src_a);
    const unsigned ntma = __popc(__ballot_sync(0xffffffffu, tma_a));
    if (lane == 0) mbar_arrive_expect_tx(bar, ntma * A_BYTES);
    __syncwarp();
    if (tma_a) {
        fence_proxy_async();
        bulk_load_l2(a_st + lane * GE::CS, src_a, A_BYTES, bar, l2_kind(l2, k));
    }
    // fallback chunk-stages
    unsigned slow = __ballot_sync(0xffffffffu, mine && !tma_a);
    while (slow) {
        const int ch = __ffs(slow) - 1;
        slow &= slow - 1;
        const int64_t abase = __shfl_sync(0xffffffffu, my_abase, ch);
        const int m = __shfl_sync(0xffffffffu, my_m, ch);
        const int nv = __shfl_sync(0xffffffffu, nvalid, ch);
        S *dst = a_st + ch * GE::CS;
        if (exact) {
            const S *s0 = a + abase + (int64_t)roff * MP;
            for (int idx = lane; idx < SRS * MP; idx += 32) {
                const bool v = idx < nv * MP;
                cp_async<sizeof(S)>(dst + idx, v ? s0 + idx : a, v ? (int)sizeof(S) : 0);
            }
        } else {
            // padded order: the m real coefficients of every row; the padded
            // columns were zeroed once and are never written
            for (int r = 0; r < SRS; ++r) {
                if (lane < m) {
                    const bool v = r < nv;
                    const S *s0 = v ? a + abase + (int64_t)(roff + r) * m + lane : a;
                    cp_async<sizeof(S)>(dst + r * MP + lane, s0, v ? (int)sizeof(S) : 0);
                }
            }
        }
    }
    cp_async_commit();
}

// Generated stage k (SRC_CONST / SRC_FRAMES): the warp writes the CPW x SRS
// coefficient rows itself, then completes the stage's mbarrier phase with no
// bytes in flight, so the consumer waits exactly as for a copied stage.
template <int MP, typename GE, bool BWD, int SRC>
__device__ __forceinline__ void k1_gen_stage(float *a_st, uint64_t *bar, const CoefSrc &cs, int M, int L, int k,
                                             int lane, int64_t my_b, int64_t my_t0, int my_valid) {
    constexpr int CPW = GE::CPW;
    const int roff = BWD ? L - (k + 1) * SRS : k * SRS;
    static_assert((CPW * SRS) % 32 == 0, "whole rows per lane");
#pragma unroll 1
    for (int e = lane; e < CPW * SRS; e += 64) {
        if (e + 32 >= CPW * SRS) {  // an odd row count per lane: the last one alone
            const int ch = e / SRS, r = e % SRS;
            const int64_t b = __shfl_sync(0xffffffffu, my_b, ch);
            const int64_t t0 = __shfl_sync(0xffffffffu, my_t0, ch);
            const int valid = __shfl_sync(0xffffffffu, my_valid, ch);
            gen_row<MP, SRC>(cs, M, b, t0 + roff + r, roff + r < valid, a_st + ch * GE::CS + r * MP);
            continue;
        }
        const int ch0 = e / SRS, r0 = e % SRS, ch1 = (e + 32) / SRS, r1 = (e + 32) % SRS;
        const int64_t b0 = __shfl_sync(0xffffffffu, my_b, ch0), b1 = __shfl_sync(0xffffffffu, my_b, ch1);
        const int64_t s0 = __shfl_sync(0xffffffffu, my_t0, ch0), s1 = __shfl_sync(0xffffffffu, my_t0, ch1);
        const int n0 = __shfl_sync(0xffffffffu, my_valid, ch0), n1 = __shfl_sync(0xffffffffu, my_valid, ch1);
        gen_rows2<MP, SRC>(cs, M, b0, s0 + roff + r0, roff + r0 < n0, a_st + ch0 * GE::CS + r0 * MP, b1,
                           s1 + roff + r1, roff + r1 < n1, a_st + ch1 * GE::CS + r1 * MP);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(bar, 0u);
    cp_async_commit();
}

// Generated stage k (forward) of the warp's chunks out to the row cache:
// one bulk store per full, aligned chunk-stage, coalesced plain stores for
// the rest; every lane then commits one bulk group, so a later
// bulk_wait_read_prev() in each lane waits for this stage's store only once
// the next one has been issued.
template <int MP, typename GE>
__device__ __forceinline__ void k1_cache_stage(float *__restrict__ cache, const float *a_st, int k, int lane,
                                               int64_t my_base, int my_valid) {
    constexpr int CPW = GE::CPW;
    constexpr unsigned BYTES = SRS * MP * sizeof(float);
    const int roff = k * SRS;
    int nvalid = my_valid - roff;
    nvalid = nvalid < 0 ? 0 : (nvalid > SRS ? SRS : nvalid);
    const bool mine = lane < CPW;
    float *dst = cache + (my_base + roff) * (int64_t)MP;
    const bool bulk = mine && nvalid == SRS && aligned16(dst);
    // the generated rows (written by every lane) before the async proxy reads them
    fence_proxy_async();
    __syncwarp();
    if (bulk) bulk_store(dst, a_st + lane * GE::CS, BYTES);
    unsigned slow = __ballot_sync(0xffffffffu, mine && !bulk && nvalid > 0);
    while (slow) {
        const int ch = __ffs(slow) - 1;
        slow &= slow - 1;
        const int64_t base = __shfl_sync(0xffffffffu, my_base, ch);
        const int nv = __shfl_sync(0xffffffffu, nvalid, ch);
        float *d = cache + (base + roff) * (int64_t)MP;
        const float *src = a_st + ch * GE::CS;
        for (int idx = lane; idx < nv * MP; idx += 32) d[idx] = src[idx];
    }
    bulk_commit();
}

// Input samples of stage k for the warp's chunks into the stage's input slot
// (16-byte cp.async pieces, element copies with zero fill at a ragged or
// misaligned piece); the coefficient issue that follows commits the group.
template <typename S, typename GE, bool BWD>
__device__ __forceinline__ void k1_stage_inputs(S *u_st, const S *__restrict__ u, int L, int k, int lane,
                                                int64_t my_base, int my_valid) {
    constexpr int E = 16 / (int)sizeof(S);  // samples per piece
    constexpr int PPC = SRS / E;             // pieces per chunk-stage
    constexpr int NP = GE::CPW * PPC;
    const int roff = BWD ? L - (k + 1) * SRS : k * SRS;
#pragma unroll
    for (int p0 = 0; p0 < NP; p0 += 32) {
        const int pc = p0 + lane;
        const int ch = pc < NP ? pc / PPC : 0;
        const int64_t base = __shfl_sync(0xffffffffu, my_base, ch);
        const int valid = __shfl_sync(0xffffffffu, my_valid, ch);
        if (pc < NP) {
            const int r = (pc % PPC) * E;  // first row of the piece
            S *dst = u_st + ch * SRS + r;
            const S *src = u + base + roff + r;
            if (roff + r + E <= valid && aligned16(src)) {
                cp_async<16>(dst, src, 16);
            } else {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const bool v = roff + r + i < valid;
                    cp_async<sizeof(S)>(dst + i, v ? src + i : u, v ? (int)sizeof(S) : 0);
                }
            }
        }
    }
}

// The body of k1_summary for block `bid` of its launch (a mixed-order launch
// runs the bodies of several orders, each block one of them).
template <typename S, int MP, int G, int R, bool BWD, int SRC = SRC_STREAM>
__device__ __forceinline__ void k1_body(int64_t bid, Batch bt, int M, int L, int64_t NQ, const S *__restrict__ a,
                                        const S *__restrict__ u, S *__restrict__ Y, int exact_flag,
                                        unsigned *__restrict__ scan_cnt, int n_cnt, int l2, int *__restrict__ status,
                                        const CoefSrc &cs) {
    static_assert(SRC == SRC_STREAM || sizeof(S) == 4, "generated coefficient rows are FP32");
    using GE = SumGeo<S, MP, G, R>;
    constexpr int CPW = GE::CPW, NS = GE::NS, WIN = MP + SR;
    constexpr int RS = YGeo<S, MP>::RS, YS = YGeo<S, MP>::YS;
    extern __shared__ __align__(128) unsigned char k1_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    if (bt.off != nullptr) pdl_wait();  // the chunk tables come from the kernel before
    NQ = batch_chunks(bt, NQ);
    const int64_t q0 = (bid * wpb + warp) * CPW;
    if (q0 >= NQ) return;
    const bool exact = exact_flag != 0;
    unsigned char *wbase = k1_smem + (size_t)warp * GE::WARP_BYTES;
    S *a_buf = reinterpret_cast<S *>(wbase);      // [NS][A_STAGE]
    S *u_buf = a_buf + NS * GE::A_STAGE;           // [NS][U_STAGE]
    uint64_t *bars = reinterpret_cast<uint64_t *>(u_buf + NS * GE::U_STAGE);
    if (!exact) {
        for (int idx = lane; idx < NS * GE::A_STAGE; idx += 32) a_buf[idx] = S(0);
    }
    if (lane == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    // lane ch < CPW describes chunk q0 + ch: its first row and valid rows
    int64_t my_base = 0, my_b = 0, my_t0 = 0, my_abase = 0;
    int my_valid = 0, my_m = M;
    if (lane < CPW && q0 + lane < NQ) {
        const ChunkPos cp = chunk_pos(bt, q0 + lane, L, M);
        my_base = cp.base;
        my_valid = cp.valid;
        my_b = cp.g;
        my_t0 = cp.c * (int64_t)L;
        my_abase = cp.abase;
        my_m = cp.m;
        if (bt.off != nullptr && !index_ok(cp.b >= 0 && cp.b < bt.n && q0 + lane < __ldg(bt.cstart + cp.b + 1),
                                           CHK_CHUNK_SIGNAL, status))
            my_valid = 0;  // stage nothing
    }
    // stage k of the coefficient rows into ring slot `slot`
    auto stage = [&](int slot, int k) {
        k1_stage_inputs<S, GE, BWD>(u_buf + slot * GE::U_STAGE, u, L, k, lane, my_base, my_valid);
        if constexpr (SRC == SRC_STREAM)
            k1_issue_stage<S, MP, GE, BWD>(a_buf + slot * GE::A_STAGE, bars + slot, a, L, k, lane, my_abase, my_m,
                                           my_valid, exact, l2);
        else {
            float *st_rows = reinterpret_cast<float *>(a_buf + slot * GE::A_STAGE);
            // the slot's rows of two stages back have left for the cache
            if (!BWD && cs.cache != nullptr) bulk_wait_read_prev();
            k1_gen_stage<MP, GE, BWD, SRC>(st_rows, bars + slot, cs, M, L, k, lane, my_b, my_t0, my_valid);
            if (!BWD && cs.cache != nullptr) k1_cache_stage<MP, GE>(cs.cache, st_rows, k, lane, my_base, my_valid);
        }
    };
    const int grp = lane / G, g = lane % G;
    const int nblk = L / SRS;

    // forward window: h[k][MP - i] = s(t - i) at a block start; backward
    // window: h[k][j - 1] = q_j at a block start.  For FP32 with an even R,
    // recursions 2p and 2p+1 share one register pair per window entry (hp)
    // and step together through packed fmas: they use the same coefficient.
    constexpr bool PK = sizeof(S) == 4 && R % 2 == 0;
    constexpr int RH = PK ? R / 2 : 1;
    S h[PK ? 1 : R][PK ? 1 : WIN];
    unsigned long long hp[RH][PK ? WIN : 1];
    auto unit_of = [&](int k, int m) -> S {
        const int r = g * R + k;
        const int unit = BWD ? r - 1 : MP - r;
        return (r >= 1 && r <= MP && m == unit) ? S(1) : S(0);
    };
    if constexpr (PK) {
#pragma unroll
        for (int p2 = 0; p2 < RH; ++p2)
#pragma unroll
            for (int m = 0; m < WIN; ++m) hp[p2][m] = f2_pack((float)unit_of(2 * p2, m), (float)unit_of(2 * p2 + 1, m));
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int m = 0; m < WIN; ++m) h[k][m] = unit_of(k, m);
    }
    const S flag0 = (g == 0) ? S(1) : S(0);

    if constexpr (SRC == SRC_STREAM) stage(0, 0);
    pdl_wait();
    pdl_release();
    // the scan that follows counts finished groups per signal from zero
    // (warp 0 of block 0 always owns chunks, so it is still here)
    if (scan_cnt != nullptr && bid == 0 && warp == 0)
        for (int i = lane; i < n_cnt * kCntStride; i += 32) scan_cnt[i] = 0u;
    // generated rows may read frames an earlier kernel wrote: after the wait
    if constexpr (SRC != SRC_STREAM) stage(0, 0);
#pragma unroll 1
    for (int k = 0; k < nblk; ++k) {
        const int slot = k & 1;
        const bool more = k + 1 < nblk;
        if (more) {
            // the other slot was consumed in the previous iteration
            stage(slot ^ 1, k + 1);
        } else {
            cp_async_commit();
        }
        cp_async_wait<1>();
        if (!mbar_wait_warp(bars + slot, (k >> 1) & 1, kWaitLimit)) {
            // a bulk copy never completed: record it, give the copies this
            // warp still has in flight (the late one and the next stage's) a
            // bounded chance to land, and leave
            if (lane == 0) atomicExch(status, DEV_TIMEOUT_TMA);
            mbar_wait_warp(bars + slot, (k >> 1) & 1, kWaitLimit);
            if (more) mbar_wait_warp(bars + (slot ^ 1), ((k + 1) >> 1) & 1, kWaitLimit);
            cp_async_wait<0>();
            if (SRC != SRC_STREAM && cs.cache != nullptr) bulk_wait_all();
            return;
        }
        __syncwarp();
        const S *arow = a_buf + slot * GE::A_STAGE + grp * GE::CS;
        const S *urow = u_buf + slot * GE::U_STAGE + grp * SRS;
        // one SR-row block per iteration (kept rolled: the unrolled block is
        // large and the instruction cache holds one)
#pragma unroll 1
        for (int cb = 0; cb < SRS / SR; ++cb) {
            // forward: rows cb*SR + j; backward: the stage's rows in reverse
            const int rb = BWD ? (SRS / SR - 1 - cb) * SR : cb * SR;
#pragma unroll
            for (int j = 0; j < SR; ++j) {
                const int row = BWD ? rb + SR - 1 - j : rb + j;
                S c[MP];
                load_row_smem<S, MP>(c, arow + row * MP);
                const S uu = flag0 * urow[row];
                if constexpr (PK) {
                    // the input drives recursion 0 only: the low half of pair 0
                    const unsigned long long u0 = f2_pack((float)uu, 0.f);
                    if constexpr (BWD) {
                        const unsigned long long one = f2_pack(1.f, 1.f), zero = 0ull;
                        unsigned long long yp[RH];
#pragma unroll
                        for (int p2 = 0; p2 < RH; ++p2) yp[p2] = f2_fma(one, hp[p2][j], p2 == 0 ? u0 : zero);
#pragma unroll
                        for (int i = 1; i < MP; ++i) {
                            const unsigned long long nc = f2_pack(-(float)c[i - 1], -(float)c[i - 1]);
#pragma unroll
                            for (int p2 = 0; p2 < RH; ++p2) hp[p2][j + i] = f2_fma(nc, yp[p2], hp[p2][j + i]);
                        }
                        const unsigned long long nl = f2_pack(-(float)c[MP - 1], -(float)c[MP - 1]);
#pragma unroll
                        for (int p2 = 0; p2 < RH; ++p2) hp[p2][j + MP] = f2_fma(nl, yp[p2], zero);
                    } else {
                        unsigned long long accp[RH];
#pragma unroll
                        for (int p2 = 0; p2 < RH; ++p2) accp[p2] = p2 == 0 ? u0 : 0ull;
#pragma unroll
                        for (int i = MP; i >= 1; --i) {
                            const unsigned long long nc = f2_pack(-(float)c[i - 1], -(float)c[i - 1]);
#pragma unroll
                            for (int p2 = 0; p2 < RH; ++p2) accp[p2] = f2_fma(nc, hp[p2][MP + j - i], accp[p2]);
                        }
#pragma unroll
                        for (int p2 = 0; p2 < RH; ++p2) hp[p2][MP + j] = accp[p2];
                    }
                } else if constexpr (BWD) {
                    S y[R];
#pragma unroll
                    for (int kk = 0; kk < R; ++kk) y[kk] = ((kk == 0) ? uu : S(0)) + h[kk][j];
#pragma unroll
                    for (int i = 1; i < MP; ++i)
#pragma unroll
                        for (int kk = 0; kk < R; ++kk) h[kk][j + i] = fma(-c[i - 1], y[kk], h[kk][j + i]);
#pragma unroll
                    for (int kk = 0; kk < R; ++kk) h[kk][j + MP] = -c[MP - 1] * y[kk];
                } else {
                    S acc[R];
#pragma unroll
                    for (int kk = 0; kk < R; ++kk) acc[kk] = (kk == 0) ? uu : S(0);
#pragma unroll
                    for (int i = MP; i >= 1; --i)
#pragma unroll
                        for (int kk = 0; kk < R; ++kk) acc[kk] = fma(-c[i - 1], h[kk][MP + j - i], acc[kk]);
#pragma unroll
                    for (int kk = 0; kk < R; ++kk) h[kk][MP + j] = acc[kk];
                }
            }
            if constexpr (PK) {
#pragma unroll
                for (int p2 = 0; p2 < RH; ++p2)
#pragma unroll
                    for (int m = 0; m < MP; ++m) hp[p2][m] = hp[p2][m + SR];
            } else {
#pragma unroll
                for (int kk = 0; kk < R; ++kk) slide<S, MP, WIN>(h[kk]);
            }
        }
        __syncwarp();
    }
    // the ring's last rows have left for the cache before it is reused
    if (SRC != SRC_STREAM && cs.cache != nullptr) bulk_wait_all();
    // end states: the warp's CPW maps (consecutive in Y) are staged in its
    // now idle stage ring, then written as one run of 16-byte stores
    constexpr bool STAGED = (size_t)CPW * YS * sizeof(S) <= GE::RING_BYTES;
    const int64_t q = q0 + grp;
    S *ys = STAGED ? a_buf : Y + q0 * YS;
    if (STAGED || q < NQ) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int r = g * R + k;
            if (r <= MP) {
                S *row = ys + grp * YS + r * RS;
                auto hv = [&](int m) -> S {
                    if constexpr (PK) return (S)((k & 1) ? f2_hi(hp[k / 2][m]) : f2_lo(hp[k / 2][m]));
                    else return h[k][m];
                };
#pragma unroll
                for (int j = 0; j < MP; ++j) row[j] = BWD ? hv(j) : hv(MP - 1 - j);
#pragma unroll
                for (int j = MP; j < RS; ++j) row[j] = S(0);
            }
        }
    }
    if constexpr (STAGED) {
        __syncwarp();
        const int nq = (int)(NQ - q0 < CPW ? NQ - q0 : CPW);
        const int n16 = (int)((size_t)nq * YS * sizeof(S) / 16);
        const float4 *src = reinterpret_cast<const float4 *>(ys);
        float4 *dst = reinterpret_cast<float4 *>(Y + q0 * YS);
        for (int i = lane; i < n16; i += 32) dst[i] = src[i];
    }
}

template <typename S, int MP, int G, int R, bool BWD, int SRC = SRC_STREAM>
__global__ void __launch_bounds__(256, 1)
    k1_summary(Batch bt, int M, int L, int64_t NQ, const S *__restrict__ a, const S *__restrict__ u,
               S *__restrict__ Y, int exact_flag, unsigned *__restrict__ scan_cnt, int n_cnt, int l2,
               int *__restrict__ status, CoefSrc cs) {
    k1_body<S, MP, G, R, BWD, SRC>(blockIdx.x, bt, M, L, NQ, a, u, Y, exact_flag, scan_cnt, n_cnt, l2, status, cs);
}

// ---------------------------------------------------------------------------
// One recursion per lane over its chunk ("lane per chunk"): a warp owns 32
// consecutive chunks.  Each lane has a private ring of two stages of SRS
// coefficient rows; a full, aligned lane-stage arrives by one bulk copy
// completing on the warp's per-stage mbarrier, others by cp.async with zero
// fill.  Input samples are loaded into registers one stage ahead.
//   FWD_RERUN: start from X[q] (or zi / zero), write s.  X rows have stride
//              xs: MP for the scan's states, M for checkpoints.
//   BWD_ZERO:  adjoint from zero state, store the end state to Z[q].
//   BWD_RERUN: adjoint from W[q], write ge; chunk 0 also writes gzi.
//   BWD_GRAD:  BWD_RERUN that also writes Eq. 12's ga(t) = -ge(t) s(t-i)
//              (exact rows only, M == MP).  The adjoint uses row a(t) up at
//              step t, so the lane writes ga(t) over it in its ring and the
//              finished stage leaves by one bulk store.
// A launch with one chunk per signal (L >= T) is the plain sequential filter.
// With `reverse` set, warps walk the chunks from the end, so a pass right
// after another over the same rows starts with the rows that pass loaded
// last (most likely still in L2).
// ---------------------------------------------------------------------------
enum { FWD_RERUN = 0, BWD_ZERO = 1, BWD_RERUN = 2, BWD_GRAD = 3 };

// Defect correction of the chunked scan (FP32).  The chunk transfers P_c
// come from M recursions in FP32, whose rounding on resonant filters is
// amplified along the chain of chunk states well beyond the rounding of
// the sequential recursion.  One correction sweep removes that excess:
//   pass 1  the re-run from the scanned state x_c reaches the chunk's end
//           state by the sequential recursion itself; its defect against
//           the scanned state of the next chunk is d_c (forward:
//           d_c = x_end(c) - x_{c+1}; adjoint: d_c = w_start(c) - w_{c-1});
//   scan    the error of the scanned states obeys the same linear
//           recurrence with the defects as its input,
//           e_{c+1} = P_c e_c + d_c  (adjoint: e_{c-1} = P_c^T e_c + d_c);
//   pass 2  every chunk whose correction is not negligible, at its start
//           or carried through the chunk (max(|e_c|, |P_c e_c|) >
//           kFixTheta * max_t |out(t)| of its signal), re-runs from
//           x_c + e_c and writes its outputs again.
// The error of e_c itself is second order (e_c is already a small
// multiple of the rounding), so the result has the rounding of the
// sequential recursion.  A signal whose outputs are not finite is never
// corrected (the comparisons fail), and neither is a chunk whose
// correction is below the threshold: skipping it changes the result by
// less than the threshold times the chunk's gain.  The decisions depend on
// the signal's own values only, so batching leaves them unchanged.
constexpr float kFixTheta = 2.0e-6f;
constexpr int kScaleWord = 16;  // per-signal max |output| (float bits) in the signal's counter line

template <typename S> struct Fix {
    S *D = nullptr;             // pass 1: defect of every chunk, stride ZS (zero where none)
    const S *E = nullptr;       // pass 2: correction of every chunk's incoming state, stride MP
    S *ckpt = nullptr;          // pass 2, forward: corrected incoming state of re-run chunks [q][M]
    unsigned *scale = nullptr;  // counter lines; word kScaleWord of line b = max |out| of signal b
    // pass 2: the chunks to re-run, in the order the correction scan listed
    // them, and their count (the word after the signals' counter lines)
    const int *list = nullptr;
    const unsigned *list_n = nullptr;
};

__device__ __forceinline__ float scale_of(const unsigned *scale, int64_t b) {
    return __uint_as_float(__ldcg(scale + b * kCntStride + kScaleWord));
}
// max of |y| that keeps a NaN (fmax would drop it): a signal with any
// non-finite output gets an infinite scale and is never corrected
template <typename S> __device__ __forceinline__ S abs_max_nan(S m, S y) {
    const S a = fabs(y);
    return (a > m || a != a) ? a : m;
}

constexpr int kRecChunks = 16;  // chunks per warp (lanes 0 .. kRecChunks-1 own one each)
// chunks per warp when the rows are generated: half the shared ring per
// warp, so twice the warps fit on an SM to hide the generator's latency
constexpr int kRecChunksGen = 4;
template <int SRC> struct RecChunks {
    static constexpr int N = SRC == SRC_STREAM ? kRecChunks : kRecChunksGen;
};

template <typename S, int MP, int RC = kRecChunks> struct RecGeo {
    static constexpr int NS = 2;                                    // stages per lane ring
    static constexpr int A_ST = SRS * MP;                           // coefficient elements per lane-stage
    static constexpr int RAW = (NS * A_ST * (int)sizeof(S)) / 4;    // words per lane
    // lane stride in words: an odd multiple of 4, so the 16-byte row loads of
    // a quarter warp hit distinct bank quads
    static constexpr int LW = ((RAW + 3) / 4) % 2 == 1 ? ((RAW + 3) / 4) * 4 : ((RAW + 3) / 4 + 1) * 4;
    static constexpr size_t SMEM = size_t(RC) * LW * 4 + NS * 8;
    // BWD_GRAD: plus one lane-stage that the lanes without a chunk read
    // (owners write gradient rows over their own rings as they go)
    static constexpr size_t SMEM_GA = SMEM + size_t(A_ST) * sizeof(S);
    static_assert((A_ST * sizeof(S)) % 16 == 0, "16-byte lane stages");
    static_assert((LW * 4) % 16 == 0, "16-byte lane ring alignment");
    static_assert(NS * A_ST * sizeof(S) <= size_t(LW) * 4, "lane ring fits its stride");
};

template <typename S, int MP, bool EXACT, bool BWD>
__device__ __forceinline__ void rec_issue_stage(S *a_st, uint64_t *bar, const S *__restrict__ a, int M, int L, int s,
                                                bool active, int64_t abase, int n, int l2, bool owner) {
    constexpr unsigned A_BYTES = SRS * MP * sizeof(S);
    const int roff = BWD ? L - (s + 1) * SRS : s * SRS;
    int nv = n - roff;
    nv = nv < 0 ? 0 : (nv > SRS ? SRS : nv);
    if (!active) nv = 0;
    const S *src_a = a + abase + (int64_t)roff * M;
    const bool tma_a = EXACT && nv == SRS && aligned16(src_a);
    const unsigned ntma = __popc(__ballot_sync(0xffffffffu, tma_a));
    if ((threadIdx.x & 31) == 0) mbar_arrive_expect_tx(bar, ntma * A_BYTES);
    __syncwarp();
    if (tma_a) {
        fence_proxy_async();
        bulk_load_l2(a_st, src_a, A_BYTES, bar, l2_kind(l2, s));
    } else if (!owner) {
        // no ring of its own: writes nothing
    } else if (EXACT) {
        for (int idx = 0; idx < SRS * MP; ++idx) {
            const bool v = idx < nv * MP;
            cp_async<sizeof(S)>(a_st + idx, v ? src_a + idx : a, v ? (int)sizeof(S) : 0);
        }
    } else {
        for (int r = 0; r < SRS; ++r)
            for (int i = 0; i < M; ++i) {
                const bool v = r < nv;
                cp_async<sizeof(S)>(a_st + r * MP + i, v ? src_a + (int64_t)r * M + i : a, v ? (int)sizeof(S) : 0);
            }
    }
    cp_async_commit();
}

// Generated stage s (SRC_CONST / SRC_FRAMES) for all RC chunks of the warp:
// all 32 lanes write rows (chunk e / SRS, row e % SRS) into the owner lanes'
// rings, then the stage's mbarrier phase completes with no bytes in flight.
template <int MP, bool BWD, int SRC, int RC>
__device__ __forceinline__ void rec_gen_stage(unsigned char *smem, int slot, uint64_t *bar, const CoefSrc &cs, int M,
                                              int L, int s, int lane, int64_t b, int64_t t0, int n, bool active) {
    using RG = RecGeo<float, MP, RC>;
    const int roff = BWD ? L - (s + 1) * SRS : s * SRS;
    static_assert((RC * SRS) % 64 == 0, "rows of a stage come in pairs per lane");
    const int actv = active ? 1 : 0;
#pragma unroll 1
    for (int e = lane; e < RC * SRS; e += 64) {
        const int ch0 = e / SRS, r0 = e % SRS, ch1 = (e + 32) / SRS, r1 = (e + 32) % SRS;
        const int64_t b0 = __shfl_sync(0xffffffffu, b, ch0), b1 = __shfl_sync(0xffffffffu, b, ch1);
        const int64_t s0 = __shfl_sync(0xffffffffu, t0, ch0), s1 = __shfl_sync(0xffffffffu, t0, ch1);
        const int n0 = __shfl_sync(0xffffffffu, n, ch0), n1 = __shfl_sync(0xffffffffu, n, ch1);
        const bool a0 = __shfl_sync(0xffffffffu, actv, ch0) != 0, a1 = __shfl_sync(0xffffffffu, actv, ch1) != 0;
        float *ring0 = reinterpret_cast<float *>(smem + (size_t)ch0 * RG::LW * 4) + slot * RG::A_ST;
        float *ring1 = reinterpret_cast<float *>(smem + (size_t)ch1 * RG::LW * 4) + slot * RG::A_ST;
        gen_rows2<MP, SRC>(cs, M, b0, s0 + roff + r0, a0 && roff + r0 < n0, ring0 + r0 * MP, b1, s1 + roff + r1,
                           a1 && roff + r1 < n1, ring1 + r1 * MP);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(bar, 0u);
    cp_async_commit();
}

template <typename S, bool BWD>
__device__ __forceinline__ void rec_load_inputs(S (&uv)[SRS], const S *__restrict__ u, int L, int s, bool active,
                                                int64_t base, int n) {
    const int roff = BWD ? L - (s + 1) * SRS : s * SRS;
    const S *src = u + base + roff;
    if (active && roff + SRS <= n && aligned16(src)) {
        // a full, aligned stage: 16-byte loads
        if constexpr (sizeof(S) == 4) {
#pragma unroll
            for (int k = 0; k < SRS / 4; ++k) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + k);
                uv[4 * k] = v.x;
                uv[4 * k + 1] = v.y;
                uv[4 * k + 2] = v.z;
                uv[4 * k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < SRS / 2; ++k) {
                const double2 v = __ldg(reinterpret_cast<const double2 *>(src) + k);
                uv[2 * k] = v.x;
                uv[2 * k + 1] = v.y;
            }
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < SRS; ++r) uv[r] = (active && roff + r < n) ? __ldg(src + r) : S(0);
}

// A lane's outputs of one stage (rows roff .. roff + SRS - 1 of its chunk,
// the first nv of them valid) from registers to memory: 16-byte stores when
// the stage is full and aligned.
template <typename S>
__device__ __forceinline__ void rec_store_outputs(S *dst, const S (&yv)[SRS], int nv) {
    if (nv == SRS && aligned16(dst)) {
        if constexpr (sizeof(S) == 4) {
#pragma unroll
            for (int k = 0; k < SRS / 4; ++k)
                reinterpret_cast<float4 *>(dst)[k] = make_float4(yv[4 * k], yv[4 * k + 1], yv[4 * k + 2], yv[4 * k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < SRS / 2; ++k) reinterpret_cast<double2 *>(dst)[k] = make_double2(yv[2 * k], yv[2 * k + 1]);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < SRS; ++r)
        if (r < nv) dst[r] = yv[r];
}

// The body of k_rec for block `bid` of `nblocks` (a mixed-order launch runs
// the bodies of several orders, each block one of them).
template <typename S, int MP, bool EXACT, int MODE, int SRC = SRC_STREAM, int RC = RecChunks<SRC>::N>
__device__ __forceinline__ void rec_body(int64_t bid, int64_t nblocks, Batch bt, int M, int L, int64_t NQ,
                                         const S *__restrict__ a, const S *__restrict__ u, const S *__restrict__ Xin,
                                         const S *__restrict__ zi, S *__restrict__ out, S *__restrict__ Zout,
                                         S *__restrict__ gzi, int reverse, unsigned *__restrict__ scan_cnt, int n_cnt,
                                         int l2, int xs, int *__restrict__ status, const CoefSrc &cs,
                                         const S *__restrict__ sfw, S *__restrict__ ga, const Fix<S> &fx) {
    static_assert(SRC == SRC_STREAM || sizeof(S) == 4, "generated coefficient rows are FP32");
    static_assert(RC >= 1 && RC <= 32, "chunks per warp");
    using RG = RecGeo<S, MP, RC>;
    constexpr int NS = RG::NS, WIN = MP + SR;
    constexpr bool BWD = MODE != FWD_RERUN;
    constexpr bool GA = MODE == BWD_GRAD;  // also Eq. 12, from s (sfw) and zi
    constexpr bool RERUN_B = MODE == BWD_RERUN || GA;
    static_assert(!GA || (EXACT && SRC == SRC_STREAM), "fused gradient rows need exact streamed rows");
    extern __shared__ __align__(128) unsigned char rec_smem[];
    const int lane = threadIdx.x & 31;
    // pass 2 of the defect correction walks its list from the first block,
    // so the few warps with work are the first to be scheduled
    const int64_t blk = (reverse && fx.E == nullptr) ? nblocks - 1 - bid : bid;
    // lanes past RC own no chunk; they read (and never write) the ring of
    // lane lane % RC so every shared access stays in range
    const bool owner = lane < RC;
    // the chunk tables (varlen) and the corrections (pass 2 of the defect
    // correction) come from the kernel before
    if (bt.off != nullptr || fx.E != nullptr) pdl_wait();
    NQ = batch_chunks(bt, NQ);
    int64_t q = blk * RC + lane;
    bool active = owner && q < NQ;
    if (fx.E != nullptr) {
        // pass 2: the warp takes RC entries of the list of chunks to re-run
        const int64_t n_list = (int64_t)__ldcg(fx.list_n);
        if (blk * RC >= n_list) return;
        active = owner && q < n_list;
        q = active ? (int64_t)__ldcg(fx.list + q) : 0;
        if (active && !index_ok(q >= 0 && q < NQ, CHK_FIX_LIST_ENTRY, status)) active = false;
    }
    S *a_ring = reinterpret_cast<S *>(rec_smem + (size_t)(lane % RC) * RG::LW * 4);  // [NS][SRS*MP]
    uint64_t *bars = reinterpret_cast<uint64_t *>(rec_smem + (size_t)RC * RG::LW * 4);
    // BWD_GRAD: lanes without a chunk read this never-written stage instead
    const S *idle_rows = reinterpret_cast<const S *>(rec_smem + (size_t)RC * RG::LW * 4 + NS * 8);
    if (!EXACT && owner) {
        for (int j = 0; j < NS * RG::A_ST; ++j) a_ring[j] = S(0);
    }
    if (lane == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    // b: the chunk's signal (in its class, for mixed orders), g: the
    // signal's index in the batch, m: its order
    int64_t b = 0, c = 0, base = 0, g = 0, abase = 0;
    int n = 0, m = M;
    if (active) {
        const ChunkPos cp = chunk_pos(bt, q, L, M);
        b = cp.b;
        c = cp.c;
        base = cp.base;
        n = cp.valid;
        g = cp.g;
        m = cp.m;
        abase = cp.abase;
        if (bt.off != nullptr &&
            !index_ok(cp.b >= 0 && cp.b < bt.n && q < __ldg(bt.cstart + cp.b + 1), CHK_CHUNK_SIGNAL, status))
            active = false;
    }
    const int ldz = bt.ldz > 0 ? bt.ldz : M;  // initial-state stride per signal
    if (SRC == SRC_STREAM && fx.E != nullptr && active) {
        // pass 2 re-runs few chunks and is bound by the latency of its
        // stages: bring the chunk's rows and inputs into L2 at once
        l2_prefetch(a + abase, (size_t)n * m * sizeof(S));
        l2_prefetch(u + base, (size_t)n * sizeof(S));
    }
    const int nblk = L / SRS;
    auto stage = [&](int slot, int s) {
        if constexpr (SRC == SRC_STREAM)
            rec_issue_stage<S, MP, EXACT, BWD>(a_ring + slot * RG::A_ST, bars + slot, a, m, L, s, active, abase, n,
                                               l2, owner);
        else
            rec_gen_stage<MP, BWD, SRC, RC>(rec_smem, slot, bars + slot, cs, M, L, s, lane, g, c * (int64_t)L, n,
                                            active);
    };
    S ucur[SRS], unxt[SRS];
    if constexpr (SRC == SRC_STREAM) stage(0, 0);
    rec_load_inputs<S, BWD>(ucur, u, L, 0, active, base, n);
    pdl_wait();
    pdl_release();
    // a scan that follows counts finished groups per signal from zero
    if (scan_cnt != nullptr && bid == 0)
        for (int i = lane; i < n_cnt * kCntStride; i += 32) scan_cnt[i] = 0u;
    if constexpr (SRC != SRC_STREAM) stage(0, 0);
    S h[WIN];
#pragma unroll
    for (int m = 0; m < WIN; ++m) h[m] = S(0);
    S ym = S(0);  // max |output| of the chunk (defect correction's scale)
    if (active) {
        if constexpr (MODE == FWD_RERUN) {
            // h[MP - j] = s(t0 - j)
#pragma unroll
            for (int j = 1; j <= MP; ++j) {
                S v = S(0);
                if (Xin != nullptr) {
                    if (j - 1 < xs) v = Xin[q * xs + (j - 1)];
                    if (fx.E != nullptr) {
                        v += fx.E[q * MP + (j - 1)];
                        if (fx.ckpt != nullptr && j <= M) fx.ckpt[q * M + (j - 1)] = v;
                    }
                } else if (zi != nullptr && j <= m) {
                    v = zi[g * ldz + (j - 1)];
                }
                h[MP - j] = v;
            }
        } else if constexpr (RERUN_B) {
            // h[j - 1] = q_j entering from the chunk's end
            if (Xin != nullptr) {
#pragma unroll
                for (int j = 0; j < MP; ++j) {
                    if (j < xs) h[j] = Xin[q * xs + j];
                    if (fx.E != nullptr) h[j] += fx.E[q * MP + j];
                }
            }
        }
    }
#pragma unroll 1
    for (int s = 0; s < nblk; ++s) {
        const int slot = s & 1;
        const bool more = s + 1 < nblk;
        // the other slot's gradient rows (stage s - 1) have left shared memory
        if constexpr (GA) bulk_wait_read();
        if (more) {
            stage(slot ^ 1, s + 1);
            rec_load_inputs<S, BWD>(unxt, u, L, s + 1, active, base, n);
        } else {
            cp_async_commit();
        }
        cp_async_wait<1>();
        // sv[k] = s(roff - MP + k) in chunk rows: the forward output (zi
        // before the signal's start) that Eq. 12 pairs with the stage's rows
        constexpr int NV = GA ? SRS + MP - 1 : 1;
        S sv[NV];
        if constexpr (GA) {
            const int roff = L - (s + 1) * SRS;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const int l = roff - MP + k;
                const int64_t t = c * (int64_t)L + l;  // time in the signal
                S v = S(0);
                if (active && l < n) {
                    if (t >= 0) v = __ldg(sfw + base + l);
                    else if (zi != nullptr) v = __ldg(zi + g * ldz + (-t - 1));
                }
                sv[k] = v;
            }
        }
        if (!mbar_wait_warp(bars + slot, (s >> 1) & 1, kWaitLimit)) {
            // as in k1_summary: the late copy and the next stage's get a
            // bounded chance to land before the warp leaves
            if (lane == 0) atomicExch(status, DEV_TIMEOUT_TMA);
            mbar_wait_warp(bars + slot, (s >> 1) & 1, kWaitLimit);
            if (more) mbar_wait_warp(bars + (slot ^ 1), ((s + 1) >> 1) & 1, kWaitLimit);
            cp_async_wait<0>();
            if constexpr (GA) bulk_wait_all();
            return;
        }
        __syncwarp();
        S *ar = a_ring + slot * RG::A_ST;
        const S *ar_read = (GA && !owner) ? idle_rows : ar;
        const int roff = BWD ? L - (s + 1) * SRS : s * SRS;
        S yv[SRS];  // the stage's outputs, stored after the stage
#pragma unroll
        for (int cb = 0; cb < SRS / SR; ++cb) {
            const int rb = BWD ? (SRS / SR - 1 - cb) * SR : cb * SR;  // first stage row of the block
#pragma unroll
            for (int pr = 0; pr < SR / 2; ++pr) {
                // rows rb+2p, rb+2p+1; the adjoint runs the pairs, and the
                // rows inside a pair, in reverse
                const int p = BWD ? SR / 2 - 1 - pr : pr;
                const int r0 = rb + 2 * p;
                S c0[MP], c1[MP];
                load_pair_smem<S, MP>(c0, c1, ar_read + r0 * MP);
                if constexpr (MODE == FWD_RERUN) {
                    const S y0 = fwd_step_win<S, MP, WIN>(h, c0, ucur[r0], 2 * p);
                    const S y1 = fwd_step_win<S, MP, WIN>(h, c1, ucur[r0 + 1], 2 * p + 1);
                    yv[r0] = y0;
                    yv[r0 + 1] = y1;
                    if (roff + r0 < n) ym = abs_max_nan(ym, y0);
                    if (roff + r0 + 1 < n) ym = abs_max_nan(ym, y1);
                } else {
                    const S y1 = bwd_step_win<S, MP, WIN>(h, c1, ucur[r0 + 1], 2 * pr);
                    const S y0 = bwd_step_win<S, MP, WIN>(h, c0, ucur[r0], 2 * pr + 1);
                    if constexpr (RERUN_B) {
                        yv[r0 + 1] = y1;
                        yv[r0] = y0;
                        if (roff + r0 + 1 < n) ym = abs_max_nan(ym, y1);
                        if (roff + r0 < n) ym = abs_max_nan(ym, y0);
                    }
                    // both rows are in registers and no other lane reads
                    // this ring: its rows take ga
                    if constexpr (GA)
                        if (active) store_ga_pair<S, MP>(ar + r0 * MP, y0, y1, sv, r0);
                }
            }
            slide<S, MP, WIN>(h);
        }
        if constexpr (MODE == FWD_RERUN || RERUN_B) {
            if (active) {
                const int nv = n - roff < 0 ? 0 : (n - roff > SRS ? SRS : n - roff);
                rec_store_outputs<S>(out + base + roff, yv, nv);
            }
        }
        if constexpr (GA) {
            if (active) {
                int nv = n - roff;
                nv = nv < 0 ? 0 : (nv > SRS ? SRS : nv);
                S *dst = ga + abase + (int64_t)roff * MP;
                if (nv == SRS && aligned16(dst)) {
                    fence_proxy_async();
                    bulk_store(dst, ar, (unsigned)(SRS * MP * sizeof(S)));
                } else {
                    for (int i = 0; i < nv * MP; ++i) dst[i] = ar[i];
                }
            }
            bulk_commit();
        }
#pragma unroll
        for (int r = 0; r < SRS; ++r) ucur[r] = unxt[r];
        __syncwarp();
    }
    cp_async_wait<0>();
    if constexpr (GA) bulk_wait_all();
    if (!active) return;
    if constexpr (MODE == BWD_ZERO) {
        // adjoint zero-state summaries use the 16-byte stride of the scan's z
        constexpr int ZS = ((MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
#pragma unroll
        for (int j = 0; j < MP; ++j) Zout[q * ZS + j] = h[j];
    }
    if constexpr (RERUN_B) {
        if (gzi != nullptr && c == 0) {
#pragma unroll
            for (int j = 0; j < MP; ++j)
                if (j < m) gzi[g * ldz + j] = h[j];
        }
    }
    if constexpr (MODE == FWD_RERUN || RERUN_B) {
        if (fx.D != nullptr) {
            // pass 1: defect of the state this chunk hands on against the
            // scanned state of the neighbouring chunk (stride ZS, as z)
            constexpr int ZS = ((MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
            const int64_t nCb = bt.off == nullptr ? bt.nC : (int64_t)(__ldg(bt.cstart + b + 1) - __ldg(bt.cstart + b));
            const bool has = BWD ? c >= 1 : c + 1 < nCb;
            const int64_t qn = BWD ? q - 1 : q + 1;
#pragma unroll
            for (int j = 0; j < MP; ++j) {
                // forward: x_end[j] = h[MP-1-j]; adjoint: w_start[j] = h[j]
                const S hv = BWD ? h[j] : h[MP - 1 - j];
                fx.D[q * ZS + j] = has ? hv - Xin[qn * xs + j] : S(0);
            }
            const float ymf = (float)ym;
            atomicMax(fx.scale + b * kCntStride + kScaleWord, __float_as_uint(ymf <= 3.0e38f ? ymf : INFINITY));
        }
    }
}

template <typename S, int MP, bool EXACT, int MODE, int SRC = SRC_STREAM, int RC = RecChunks<SRC>::N>
__global__ void __launch_bounds__(32)
    k_rec(Batch bt, int M, int L, int64_t NQ, const S *__restrict__ a, const S *__restrict__ u,
          const S *__restrict__ Xin, const S *__restrict__ zi, S *__restrict__ out, S *__restrict__ Zout,
          S *__restrict__ gzi, int reverse, unsigned *__restrict__ scan_cnt, int n_cnt, int l2, int xs,
          int *__restrict__ status, CoefSrc cs, const S *__restrict__ sfw, S *__restrict__ ga, Fix<S> fx) {
    rec_body<S, MP, EXACT, MODE, SRC, RC>(blockIdx.x, gridDim.x, bt, M, L, NQ, a, u, Xin, zi, out, Zout, gzi,
                                          reverse, scan_cnt, n_cnt, l2, xs, status, cs, sfw, ga, fx);
}

// ---------------------------------------------------------------------------
// K2: cross-chunk scan, one cooperative launch.  Chunks are grouped G2 at a
// time by chunk index (group g = chunks [g*G2, (g+1)*G2)).  Along the chain
// the forward visits chunks and groups in increasing order, the adjoint in
// decreasing order.  Each warp owns items (b, g) and runs three phases:
//   A   fold: CH_FWD / CH_BWD compose the group's chunk maps x -> P x + y
//       into one map (Phi_g, y_g), stored in the chunk-map layout at GY;
//       CH_TRANS folds the adjoint's chunk maps w -> P^T w + z into the
//       group's zero-state adjoint zeta_g (GZ); the group's transfer is the
//       transpose of the forward's Phi_g, which GY already holds.  A
//       finished item bumps its signal's counter.
//   B1  once all nG groups of signal b are counted, the warp owning (b, 0)
//       chains the group maps (one hop each) and stores the incoming state
//       of every group in GX; then bumps the counter once more.
//   B2  each group runs one hop per chunk from its incoming state, writing
//       every chunk's incoming state X (and, in the forward, the
//       checkpoints).  A warp with a single item still holds that group's
//       chunk maps in shared memory from phase A and reads none again.
// Every warp finishes phase A before it waits, and all chain work (B1) comes
// before any B2 wait; the launch is cooperative (every block resident), so
// the waits always end; each one is also bounded.  Maps reach shared memory
// through a per-warp ring of kScanDepth slots filled by 16-byte cp.async
// copies (L2 only, so maps written by other SMs during the launch are read
// fresh).
// Chunk map layout (stride YS, rows of RS): Y[0][k] = y[k], Y[r][k] = P[k][r-1].
// ---------------------------------------------------------------------------
enum { CH_FWD = 0, CH_BWD = 1, CH_TRANS = 2, CH_FWD_FIX = 3, CH_TRANS_FIX = 4, CH_BWD_FIX = 5 };
// The _FIX modes are the correction scans of the defect correction (see
// Fix): vector scans like CH_TRANS, driven by the chunk defects (passed as
// Z) instead of zero-state summaries, through the chunk maps and group
// maps the main scan left in Y and GY (CH_FWD_FIX: the forward's maps,
// straight; CH_TRANS_FIX: the forward's maps, transposed; CH_BWD_FIX: the
// adjoint's own maps, straight, backwards).  They run right after a main
// scan of the same call, whose counters stand at nG + 1 per signal, so
// their counts start there.
template <int MODE> struct ScanMode {
    static constexpr bool REV = MODE == CH_BWD || MODE == CH_TRANS || MODE == CH_TRANS_FIX || MODE == CH_BWD_FIX;
    static constexpr bool TRANS = MODE == CH_TRANS || MODE == CH_TRANS_FIX;
    static constexpr bool VEC = MODE >= CH_TRANS;  // vector scan driven by Z, reusing GY
    static constexpr bool FIX = MODE >= CH_FWD_FIX;
};

constexpr int kScanWarps = 4;       // warps per block
constexpr int kScanDepth = 10;      // map slots per warp ring
constexpr int kScanSpin = 1 << 19;  // counter polls (~250 ns each) before a wait gives up

// Group composition on the tensor cores (FP32 data, MP >= 8): the running
// product R (MP x MP, with the accumulated response y as column MP) lives
// in a shared tile of KP rows (the product's rows, padded to the k-steps of
// an m16n8k8 MMA) and NP columns (MP+1 padded to n-tiles), row stride ST.
template <int MP> struct MmaGeo {
    static constexpr int KP = 8 * ((MP + 7) / 8);
    static constexpr int NP = 8 * ((MP + 1 + 7) / 8);
    // ST = 8 or 24 mod 32: the B-fragment loads (4 rows x 8 columns) and
    // the A loads hit 32 distinct banks
    static constexpr int ST = NP % 16 == 8 ? NP : NP + 8;
};
template <typename S, int MP> struct UseMma {
    static constexpr bool ON = sizeof(S) == 4 && MP >= 8;
};

template <typename S, int MP, int D = kScanDepth> struct ScanGeo {
    static constexpr int RS = YGeo<S, MP>::RS;
    static constexpr int YS = YGeo<S, MP>::YS;
    static constexpr int ZS = RS;         // a z vector: MP values padded to 16 bytes
    // per warp: kScanDepth map slots, kScanDepth z slots, two mbarriers,
    // two state-exchange buffers of RS values, and (FP32) the tile of the
    // running product of the tensor-core composition
    static constexpr size_t MAPS_BYTES = size_t(D) * YS * sizeof(S);
    static constexpr size_t ZS_BYTES = size_t(D) * ZS * sizeof(S);
    static constexpr size_t BAR_OFF = MAPS_BYTES + ZS_BYTES;
    static constexpr size_t XB_OFF = BAR_OFF + 16;
    static constexpr size_t R_OFF = ((XB_OFF + 2 * RS * sizeof(S) + 15) / 16) * 16;
    static constexpr size_t R_BYTES =
        UseMma<S, MP>::ON ? size_t(MmaGeo<MP>::KP) * MmaGeo<MP>::ST * sizeof(float) : 0;
    static constexpr size_t WARP_BYTES = ((R_OFF + R_BYTES + 127) / 128) * 128;
    static_assert((YS * sizeof(S)) % 16 == 0 && (ZS * sizeof(S)) % 16 == 0, "16-byte maps");
    static_assert(BAR_OFF % 16 == 0 && WARP_BYTES % 128 == 0, "aligned warp slices");
    static_assert(RS <= 32, "a padded row fits the lanes of a warp");
    static_assert(D % 2 == 0, "two halves for double buffering");
};

// x_new[lane] = p[0] + sum_{r=1..MP} p[r] * x[r-1], x held one component per lane
template <typename S, int MP>
__device__ __forceinline__ S hop(const S (&p)[MP + 1], S x, int lane) {
    S a0 = p[0], a1 = S(0), a2 = S(0), a3 = S(0);
#pragma unroll
    for (int r = 1; r <= MP; ++r) {
        const S xr = __shfl_sync(0xffffffffu, x, r - 1);
        if ((r & 3) == 0) a0 = fma(p[r], xr, a0);
        else if ((r & 3) == 1) a1 = fma(p[r], xr, a1);
        else if ((r & 3) == 2) a2 = fma(p[r], xr, a2);
        else a3 = fma(p[r], xr, a3);
    }
    return lane < MP ? (a0 + a1) + (a2 + a3) : S(0);
}

// coefficients of the lane's output component for one map held in shared
// memory: straight (x -> P x + y, map at m; with DRIVE, x -> P x + z) or
// transposed (w -> P^T w + z, P from the map at m, z at zv)
template <typename S, int MP, bool TRANS, bool DRIVE = TRANS>
__device__ __forceinline__ void map_cols(S (&p)[MP + 1], const S *m, const S *zv, int j0) {
    constexpr int RS = YGeo<S, MP>::RS;
    if constexpr (TRANS) {
        // row j0+1 holds column j0 of P: 16-byte loads along it
        constexpr int V = 16 / (int)sizeof(S);
        const S *row = m + (j0 + 1) * RS;
#pragma unroll
        for (int k = 0; k < RS; k += V) {
            if constexpr (sizeof(S) == 4) {
                const float4 v = *reinterpret_cast<const float4 *>(row + k);
                if (k + 0 < MP) p[k + 1] = v.x;
                if (k + 1 < MP) p[k + 2] = v.y;
                if (k + 2 < MP) p[k + 3] = v.z;
                if (k + 3 < MP) p[k + 4] = v.w;
            } else {
                const double2 v = *reinterpret_cast<const double2 *>(row + k);
                if (k + 0 < MP) p[k + 1] = v.x;
                if (k + 1 < MP) p[k + 2] = v.y;
            }
        }
        p[0] = zv[j0];
    } else {
#pragma unroll
        for (int r = 0; r <= MP; ++r) p[r] = m[r * RS + j0];
        if constexpr (DRIVE) p[0] = zv[j0];
    }
}

// TF32 tensor-core MMA, D += A B, m16n8k8, A row-major, B column-major.
// Fragments (g = lane / 4, t = lane % 4): a0 (g, t), a1 (g+8, t), a2 (g, t+4),
// a3 (g+8, t+4); b0 (t, g), b1 (t+4, g); d0 (g, 2t), d1 (g, 2t+1),
// d2 (g+8, 2t), d3 (g+8, 2t+1).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// x = hi + lo with hi, lo TF32 (round to nearest, ties away): the products
// hi*hi + hi*lo + lo*hi carry x's value to within about 2^-21 of it
__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// One composition step on the tensor cores: R <- P R, with y <- P y + y_c in
// column MP, for the chunk map at m (Y[0][k] = y_c[k], Y[r][k] = P[k][r-1]).
// Three TF32 products per k-step (the hi/lo split of both operands) keep
// the result within a few FP32 ulps of the FP32 composition.
template <int MP>
__device__ __forceinline__ void compose_mma(float *rs, const float *m, int lane) {
    using MG = MmaGeo<MP>;
    constexpr int RS = YGeo<float, MP>::RS, ST = MG::ST;
    constexpr int MT = (MP + 15) / 16, KT = MG::KP / 8, NT = MG::NP / 8;
    const int g = lane >> 2, t = lane & 3;
    unsigned bh[KT][NT][2], bl[KT][NT][2];
#pragma unroll
    for (int kk = 0; kk < KT; ++kk)
#pragma unroll
        for (int nn = 0; nn < NT; ++nn)
#pragma unroll
            for (int h = 0; h < 2; ++h) split_tf32(rs[(t + 4 * h + 8 * kk) * ST + g + 8 * nn], bh[kk][nn][h], bl[kk][nn][h]);
    float d[MT][NT][4];
#pragma unroll
    for (int mm = 0; mm < MT; ++mm)
#pragma unroll
        for (int nn = 0; nn < NT; ++nn)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = g + 8 * (q >> 1) + 16 * mm, col = 2 * t + (q & 1) + 8 * nn;
                d[mm][nn][q] = (col == MP && row < MP) ? m[row] : 0.f;
            }
#pragma unroll
    for (int mm = 0; mm < MT; ++mm)
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            // A = P: element (k, r) at Y[r+1][k]
            unsigned ah[4], al[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = g + 8 * (q & 1) + 16 * mm, col = t + 4 * (q >> 1) + 8 * kk;
                const float x = (row < MP && col < MP) ? m[(col + 1) * RS + row] : 0.f;
                split_tf32(x, ah[q], al[q]);
            }
#pragma unroll
            for (int nn = 0; nn < NT; ++nn) {
                mma_tf32(d[mm][nn], al, bh[kk][nn]);
                mma_tf32(d[mm][nn], ah, bl[kk][nn]);
                mma_tf32(d[mm][nn], ah, bh[kk][nn]);
            }
        }
    __syncwarp();  // every lane has read R before it is overwritten
#pragma unroll
    for (int mm = 0; mm < MT; ++mm)
#pragma unroll
        for (int nn = 0; nn < NT; ++nn)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = g + 8 * (q >> 1) + 16 * mm, col = 2 * t + (q & 1) + 8 * nn;
                if (row < MG::KP) rs[row * ST + col] = d[mm][nn][q];
            }
    __syncwarp();
}

// packed pair FMA (two IEEE fmas per instruction)
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long r, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Lanes that fold y into the composition: lane MP (idle otherwise) carries
// the accumulated response y as one more column.  MP = 32 has no spare lane
// and folds y by a separate hop chain.
template <int MP> struct YLane {
    static constexpr bool ON = MP < 32;
};

// col <- P col (+ y_c on lane MP when YLane is on) for the map at m: lane j
// holds column j of the running product, acc[k] = sum_r P[k][r-1] col[r-1]
// with rows of P read as 16-byte broadcasts; the sum runs in increasing r
// for every k, after y_c[k] on the y lane
template <typename S, int MP>
__device__ __forceinline__ void compose_step(S (&col)[MP], const S *m, int lane) {
    constexpr int RS = YGeo<S, MP>::RS;
    const bool ylane = YLane<MP>::ON && lane == MP;
    if constexpr (sizeof(S) == 4) {
        constexpr int NP = (MP + 1) / 2;  // pairs covering k < MP
        unsigned long long acc[NP];
#pragma unroll
        for (int q = 0; q + 1 < NP; q += 2) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(m + 2 * q);
            acc[q] = ylane ? v.x : 0ull;
            acc[q + 1] = ylane ? v.y : 0ull;
        }
        if constexpr (NP % 2 == 1) acc[NP - 1] = ylane ? *reinterpret_cast<const unsigned long long *>(m + 2 * (NP - 1)) : 0ull;
#pragma unroll
        for (int r = 1; r <= MP; ++r) {
            const unsigned long long xx = pack2(col[r - 1], col[r - 1]);
            const S *row = m + r * RS;
#pragma unroll
            for (int q = 0; q + 1 < NP; q += 2) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(row + 2 * q);
                acc[q] = fma2(v.x, xx, acc[q]);
                acc[q + 1] = fma2(v.y, xx, acc[q + 1]);
            }
            if constexpr (NP % 2 == 1)
                acc[NP - 1] = fma2(*reinterpret_cast<const unsigned long long *>(row + 2 * (NP - 1)), xx, acc[NP - 1]);
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float lo, hi;
            unpack2(acc[q], lo, hi);
            col[2 * q] = lo;
            if (2 * q + 1 < MP) col[2 * q + 1] = hi;
        }
    } else {
        S acc[MP];
#pragma unroll
        for (int k = 0; k < MP; ++k) acc[k] = ylane ? m[k] : S(0);
#pragma unroll
        for (int r = 1; r <= MP; ++r) {
            const S xr = col[r - 1];
            const S *row = m + r * RS;
#pragma unroll
            for (int k = 0; k + 1 < MP; k += 2) {
                const double2 v = *reinterpret_cast<const double2 *>(row + k);
                acc[k] = fma(v.x, xr, acc[k]);
                acc[k + 1] = fma(v.y, xr, acc[k + 1]);
            }
            if constexpr (MP % 2 == 1) acc[MP - 1] = fma(row[MP - 1], xr, acc[MP - 1]);
        }
#pragma unroll
        for (int k = 0; k < MP; ++k) col[k] = acc[k];
    }
}

// One hop with the state broadcast through shared memory: lane j < MP
// publishes x_j in xb (RS entries, padding zero), then every lane reads the
// whole state with 16-byte broadcasts.  xb alternates between two buffers
// from hop to hop, so one barrier per hop suffices.
template <typename S, int MP>
__device__ __forceinline__ S hop_smem(const S (&p)[MP + 1], S *xb, S x, int lane) {
    constexpr int RS = YGeo<S, MP>::RS;
    constexpr int V = 16 / (int)sizeof(S);
    if (lane < RS) xb[lane] = lane < MP ? x : S(0);
    __syncwarp();
    S a0 = p[0], a1 = S(0), a2 = S(0), a3 = S(0);
#pragma unroll
    for (int k = 0; k < RS; k += V) {
        if constexpr (sizeof(S) == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(xb + k);
            if (k + 0 < MP) a0 = fma(p[k + 1], v.x, a0);
            if (k + 1 < MP) a1 = fma(p[k + 2], v.y, a1);
            if (k + 2 < MP) a2 = fma(p[k + 3], v.z, a2);
            if (k + 3 < MP) a3 = fma(p[k + 4], v.w, a3);
        } else {
            const double2 v = *reinterpret_cast<const double2 *>(xb + k);
            if (k + 0 < MP) ((k / 2) % 2 == 0 ? a0 : a2) = fma(p[k + 1], v.x, (k / 2) % 2 == 0 ? a0 : a2);
            if (k + 1 < MP) ((k / 2) % 2 == 0 ? a1 : a3) = fma(p[k + 2], v.y, (k / 2) % 2 == 0 ? a1 : a3);
        }
    }
    return lane < MP ? (a0 + a1) + (a2 + a3) : S(0);
}

// The lane's coefficients of one map read from global memory through L2
// (another block may have written it): straight, p[r] = row r at column j0
// (row 0, the map's own constant term, unless the scan is driven by z);
// transposed, p[k+1] = row j0+1 at column k.  Driven scans set p[0] from z.
template <typename S, int MP, bool TRANS, bool VEC>
__device__ __forceinline__ void chain_map_cols(S (&p)[MP + 1], const S *__restrict__ m, int j0) {
    constexpr int RS = YGeo<S, MP>::RS;
    if constexpr (TRANS) {
        const S *row = m + (j0 + 1) * RS;
#pragma unroll
        for (int k = 0; k < RS; k += 4) {
            const float4 v = __ldcg(reinterpret_cast<const float4 *>(row + k));
            if (k + 0 < MP) p[k + 1] = v.x;
            if (k + 1 < MP) p[k + 2] = v.y;
            if (k + 2 < MP) p[k + 3] = v.z;
            if (k + 3 < MP) p[k + 4] = v.w;
        }
    } else {
#pragma unroll
        for (int r = VEC ? 1 : 0; r <= MP; ++r) p[r] = __ldcg(m + r * RS + j0);
    }
}

// A warp's map buffers: kScanDepth map slots and their z slots, filled by
// bulk (TMA) copies of contiguous runs of maps, completing on one of two
// mbarriers.  A run of up to kScanDepth maps arrives in one copy; a longer
// run streams in batches of kScanDepth/2 through the two halves.
template <typename S, int MP, int D = kScanDepth> struct ScanWarp {
    using SG = ScanGeo<S, MP, D>;
    S *maps, *zs, *xb;
    float *rs;  // tensor-core composition tile (FP32 only)
    uint64_t *bars;
    unsigned phase;  // bit h: parity of the next completion of bars[h]
    int lane;
    int *status;
    __device__ void init(unsigned char *base, int lane_, int *status_) {
        maps = reinterpret_cast<S *>(base);
        zs = reinterpret_cast<S *>(base + SG::MAPS_BYTES);
        bars = reinterpret_cast<uint64_t *>(base + SG::BAR_OFF);
        xb = reinterpret_cast<S *>(base + SG::XB_OFF);
        rs = reinterpret_cast<float *>(base + SG::R_OFF);
        phase = 0;
        lane = lane_;
        status = status_;
        if (lane == 0) {
            mbar_init(bars, 1);
            mbar_init(bars + 1, 1);
            mbar_init_fence();
        }
        __syncwarp();
    }
    __device__ const S *map(int slot) const { return maps + slot * SG::YS; }
    __device__ const S *zv(int slot) const { return zs + slot * SG::ZS; }
    // n maps (and their z vectors) from memory into slots [slot0, slot0+n)
    __device__ void issue(int slot0, int n, const S *map_src, const S *z_src, int bar) {
        __syncwarp();  // every lane's reads of the slots are done
        if (lane == 0) {
            const unsigned mb = (unsigned)(n * SG::YS * sizeof(S)), zb = z_src ? (unsigned)(n * SG::ZS * sizeof(S)) : 0u;
            fence_proxy_async();
            mbar_arrive_expect_tx(bars + bar, mb + zb);
            bulk_load(maps + slot0 * SG::YS, map_src, mb, bars + bar);
            if (z_src) bulk_load(zs + slot0 * SG::ZS, z_src, zb, bars + bar);
        }
    }
    // n z vectors alone into z slots [slot0, slot0+n)
    __device__ void issue_z(int slot0, int n, const S *z_src, int bar) {
        __syncwarp();
        if (lane == 0) {
            const unsigned zb = (unsigned)(n * SG::ZS * sizeof(S));
            fence_proxy_async();
            mbar_arrive_expect_tx(bars + bar, zb);
            bulk_load(zs + slot0 * SG::ZS, z_src, zb, bars + bar);
        }
    }
    __device__ bool wait(int bar) {
        const bool ok = mbar_wait_warp(bars + bar, (phase >> bar) & 1u, kWaitLimit);
        phase ^= 1u << bar;
        if (!ok && lane == 0) atomicExch(status, DEV_TIMEOUT_TMA);
        return ok;
    }
    // after a wait on `bar` gave up: one more bounded wait for that late copy
    __device__ void drain(int bar) { mbar_wait_warp(bars + bar, ((phase >> bar) & 1u) ^ 1u, kWaitLimit); }
};

// Runs step(i, map, z) for i = 0 .. n-1 along a contiguous run of n maps
// (memory order from map_lo / z_lo; the chain visits it backwards when
// REVR).  False when a copy never landed (status set; nothing in flight).
template <typename S, int MP, bool REVR, int DEPTH, typename Step>
__device__ __forceinline__ bool run_maps(ScanWarp<S, MP, DEPTH> &W, const S *map_lo, const S *z_lo, int n, Step step) {
    using SG = ScanGeo<S, MP, DEPTH>;
    constexpr int D = DEPTH, H = DEPTH / 2;
    if (n <= 0) return true;
    if (n <= D) {
        W.issue(0, n, map_lo, z_lo, 0);
        if (!W.wait(0)) {
            W.drain(0);
            return false;
        }
        for (int i = 0; i < n; ++i) {
            const int mi = REVR ? n - 1 - i : i;
            step(i, W.map(mi), W.zv(mi));
        }
        return true;
    }
    const int nb = (n + H - 1) / H;
    auto batch = [&](int j, int &mlo, int &cnt) {
        const int c0 = j * H;
        cnt = n - c0 < H ? n - c0 : H;
        mlo = REVR ? n - c0 - cnt : c0;
    };
    auto issue = [&](int j) {
        int mlo, cnt;
        batch(j, mlo, cnt);
        W.issue((j & 1) * H, cnt, map_lo + (size_t)mlo * SG::YS, z_lo ? z_lo + (size_t)mlo * SG::ZS : nullptr, j & 1);
    };
    issue(0);
    issue(1);
    for (int j = 0; j < nb; ++j) {
        if (!W.wait(j & 1)) {
            W.drain(j & 1);
            if (j + 1 < nb) W.wait((j + 1) & 1);  // the other half's copy, if any, is in flight
            return false;
        }
        int mlo, cnt;
        batch(j, mlo, cnt);
        for (int k = 0; k < cnt; ++k) {
            const int slot = (j & 1) * H + (REVR ? cnt - 1 - k : k);
            step(j * H + k, W.map(slot), W.zv(slot));
        }
        if (j + 2 < nb) issue(j + 2);
    }
    return true;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

// Warp-collective bounded wait until *c >= target: lane 0 polls with relaxed
// loads (sleeping about SLEEP_NS between polls), then every lane takes one
// acquire load before reading what the count guards.  After kScanSpin polls
// it records DEV_TIMEOUT_SCAN and returns false.
template <unsigned SLEEP_NS = 256>
__device__ __forceinline__ bool wait_counter(const unsigned *c, unsigned target, int lane, int *status) {
    bool ok = false;
    for (int it = 0; it < kScanSpin && !ok; ++it) {
        ok = __shfl_sync(0xffffffffu, lane == 0 ? (ld_relaxed(c) >= target) : false, 0);
        if (!ok) __nanosleep(SLEEP_NS);
    }
    (void)ld_acquire(c);
    if (!ok && lane == 0) atomicExch(status, DEV_TIMEOUT_SCAN);
    return ok;
}

// Map slots of a chain block: its whole shared memory (the slices of
// kScanWarps item warps) as one ring, an even number of slots.
template <typename S, int MP> struct ChainCap {
    using G = ScanGeo<S, MP>;
    static constexpr size_t TOTAL = size_t(kScanWarps) * G::WARP_BYTES;
    // ScanGeo<S, MP, d>::WARP_BYTES, spelled out for a run-time d
    static constexpr size_t bytes(int d) {
        return ((((size_t(d) * (G::YS + G::ZS) * sizeof(S) + 16 + 2 * G::RS * sizeof(S)) + 15) / 16 * 16 +
                 G::R_BYTES + 127) /
                128) *
               128;
    }
    static constexpr int fit(int d) { return bytes(d) <= TOTAL ? d : fit(d - 2); }
    static constexpr int N = fit(int(TOTAL / ((G::YS + G::ZS) * sizeof(S))) & ~1);
    static_assert(N >= kScanDepth, "a chain block holds at least a warp's ring");
    static_assert(ScanGeo<S, MP, N>::WARP_BYTES <= TOTAL, "the ring fits the block");
};

// Phase B1 in a chain block: warp 0 runs the chain of signals cb, cb +
// n_chain, ... with every group map the chain needs copied into the block's
// shared memory at once (one bulk copy; a chain longer than the ring
// streams through its halves).  A vector scan's group maps come from an
// earlier launch, so their copy starts before the wait for phase A and only
// the group vectors follow it.  Returns false when a wait gave up.
template <typename S, int MP, int MODE>
__device__ __forceinline__ bool chain_block(int64_t cb, int64_t n_chain, const Batch &bt, int M, int64_t items_bound,
                                            const S *GY, const S *GZ, S *GX, const S *zi, unsigned *cnt,
                                            int *status) {
    constexpr int CAP = ChainCap<S, MP>::N;
    using SG = ScanGeo<S, MP, CAP>;
    constexpr int YS = SG::YS, ZS = SG::ZS, RS = SG::RS;
    constexpr bool REV = ScanMode<MODE>::REV, TRANS = ScanMode<MODE>::TRANS, VEC = ScanMode<MODE>::VEC;
    extern __shared__ __align__(128) unsigned char k2_smem[];
    const int lane = threadIdx.x & 31;
    ScanWarp<S, MP, CAP> W;
    W.init(k2_smem, lane, status);
    const int j0 = lane < MP ? lane : 0;
    int nhop = 0;
    auto hop_step = [&](const S *m, const S *z, S x) -> S {
        S p[MP + 1];
        map_cols<S, MP, TRANS, VEC>(p, m, z, j0);
        return hop_smem<S, MP>(p, W.xb + ((nhop++) & 1) * RS, x, lane);
    };
    for (int64_t b = cb; b < bt.n; b += n_chain) {
        const SigScan sg = sig_scan(bt, b);
        const int nG = sg.nG, nh = nG - 1;
        if (nG <= 0) continue;  // an empty signal of a varlen batch has no groups
        if (!index_ok(sg.gbase >= 0 && sg.gbase + nG <= items_bound, CHK_CHAIN_GROUPS, status)) continue;
        // step n takes group gidx(n)'s incoming state through that group's
        // map: groups [gbase, gbase + nG-1) forward, [gbase + 1, gbase + nG)
        // backward, visited from the top
        auto gidx = [&](int n) -> int64_t { return sg.gbase + (REV ? nG - 1 - n : n); };
        const int64_t lo = sg.gbase + (REV ? 1 : 0);
        const bool early = VEC && nh > 0 && nh <= CAP;
        if (early) W.issue(0, nh, GY + lo * YS, nullptr, 0);
        const unsigned base = ScanMode<MODE>::FIX ? (unsigned)nG + 1u : 0u;
        if (!wait_counter(cnt + b * kCntStride, base + (unsigned)nG, lane, status)) {
            if (early) W.wait(0);
            return false;
        }
        fence_proxy_async_global();  // the group maps and vectors are read by bulk copies
        S x = S(0);
        if (MODE == CH_FWD && zi != nullptr) {
            const int64_t gs_ = global_signal(bt, b);
            const int m = bt.ord != nullptr ? __ldg(bt.ord + gs_) : M;
            if (lane < m) x = zi[gs_ * (bt.ldz > 0 ? bt.ldz : M) + lane];
        }
        if (early) {
            W.issue_z(0, nh, GZ + lo * ZS, 1);
            const bool ok0 = W.wait(0);
            const bool ok1 = W.wait(1);
            if (!ok0 || !ok1) {
                if (!ok0) W.drain(0);
                if (!ok1) W.drain(1);
                return false;
            }
            for (int n = 0; n < nh; ++n) {
                const int mi = REV ? nh - 1 - n : n;
                if (lane < ZS) GX[gidx(n) * ZS + lane] = lane < MP ? x : S(0);
                x = hop_step(W.map(mi), W.zv(mi), x);
            }
        } else {
            const bool ok = run_maps<S, MP, REV, CAP>(W, GY + lo * YS, VEC ? GZ + lo * ZS : nullptr, nh,
                                                      [&](int n, const S *m, const S *z) {
                                                          if (lane < ZS) GX[gidx(n) * ZS + lane] = lane < MP ? x : S(0);
                                                          x = hop_step(m, z, x);
                                                      });
            if (!ok) return false;
        }
        if (lane < ZS) GX[gidx(nG - 1) * ZS + lane] = lane < MP ? x : S(0);
        fence_proxy_async_global();
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(cnt + b * kCntStride, 1u);
    }
    return true;
}

// Phase B1 in a chain block with the group maps in registers: the chain
// of signal cb (one signal per chain block) is cut into kScanWarps pieces of
// up to KM steps, one per warp.  Each warp holds its pieces' map columns in
// registers (lane j: column j, MP + 1 values a map), so a hop only publishes
// and reads the state through shared memory; the state passes from warp to
// warp through an mbarrier (arrive with release, bounded wait with
// acquire).  FP32 orders up to 22 and chains of up to kScanWarps * KM steps;
// other chains take the shared-memory chain.  Returns false when a wait gave
// up.
template <typename S, int MP> struct ChainRegs {
    static constexpr int KM = 9;  // maps per warp
    // the maps take most of a thread's registers, which costs the item
    // blocks no occupancy only where shared memory already holds the scan to
    // two blocks per SM
    static constexpr bool ON = sizeof(S) == 4 && MP <= 22 && ChainCap<S, MP>::TOTAL * 3 > size_t(227) * 1024;
};

template <typename S, int MP, int MODE>
__device__ __forceinline__ bool chain_block_regs(int64_t cb, const Batch &bt, int M, int64_t items_bound,
                                                 const S *GY, const S *GZ, S *GX, const S *zi, unsigned *cnt,
                                                 int *status) {
    constexpr int KM = ChainRegs<S, MP>::KM, NW = kScanWarps;
    constexpr int YS = YGeo<S, MP>::YS, RS = YGeo<S, MP>::RS, ZS = RS;
    constexpr bool REV = ScanMode<MODE>::REV, TRANS = ScanMode<MODE>::TRANS, VEC = ScanMode<MODE>::VEC;
    extern __shared__ __align__(128) unsigned char k2_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // [NW][2][RS] the warps' publish buffers, [NW-1][RS] the hand-offs, then
    // NW-1 mbarriers (16-byte aligned)
    S *xb = reinterpret_cast<S *>(k2_smem) + (size_t)warp * 2 * RS;
    S *xh = reinterpret_cast<S *>(k2_smem) + (size_t)NW * 2 * RS;
    constexpr size_t HB_OFF = ((size_t(NW * 2 + NW - 1) * RS * sizeof(S) + 15) / 16) * 16;
    uint64_t *hb = reinterpret_cast<uint64_t *>(k2_smem + HB_OFF);
    if (threadIdx.x == 0) {
        for (int w = 0; w + 1 < NW; ++w) mbar_init(hb + w, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (cb >= bt.n) return true;
    const int64_t b = cb;
    const SigScan sg = sig_scan(bt, b);
    const int nG = sg.nG, nh = nG - 1;
    if (nG <= 0) return true;  // an empty signal of a varlen batch has no groups
    if (!index_ok(sg.gbase >= 0 && sg.gbase + nG <= items_bound, CHK_CHAIN_GROUPS, status)) return true;
    auto gidx = [&](int n) -> int64_t { return sg.gbase + (REV ? nG - 1 - n : n); };
    const int j0 = lane < MP ? lane : 0;
    // this warp's steps [n0, n1); the warp with the last step (or warp 0 for
    // a chain of one group) stores the final state and publishes
    const int n0 = warp * KM, n1 = n0 + KM < nh ? n0 + KM : nh;
    const bool mine = n0 < n1;
    const bool last = nh == 0 ? warp == 0 : (mine && n1 == nh);
    if (!mine && !last) return true;
    S pm[KM][MP + 1];
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (n0 + k < n1) {
            // a vector scan's maps come from a scan two or more launches
            // back: loaded before the waits
            if constexpr (VEC) chain_map_cols<S, MP, TRANS, true>(pm[k], GY + gidx(n0 + k) * YS, j0);
        }
    }
    // the group maps are two launches old; what follows may need the
    // previous kernel's results
    pdl_wait();
    pdl_release();
    const unsigned base = ScanMode<MODE>::FIX ? (unsigned)nG + 1u : 0u;
    // the chain is the scan's critical path: poll for its start closely
    if (!wait_counter<32>(cnt + b * kCntStride, base + (unsigned)nG, lane, status)) return false;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (n0 + k < n1) {
            if constexpr (VEC) pm[k][0] = __ldcg(GZ + gidx(n0 + k) * ZS + j0);
            else chain_map_cols<S, MP, TRANS, false>(pm[k], GY + gidx(n0 + k) * YS, j0);
        }
    }
    S x = S(0);
    if (warp == 0) {
        if (MODE == CH_FWD && zi != nullptr) {
            const int64_t gs_ = global_signal(bt, b);
            const int m = bt.ord != nullptr ? __ldg(bt.ord + gs_) : M;
            if (lane < m) x = zi[gs_ * (bt.ldz > 0 ? bt.ldz : M) + lane];
        }
    } else {
        // the state after the previous warp's steps
        if (!mbar_wait_warp(hb + (warp - 1), 0u, kWaitLimit)) {
            if (lane == 0) atomicExch(status, DEV_TIMEOUT_SCAN);
            return false;
        }
        x = lane < MP ? xh[(warp - 1) * RS + lane] : S(0);
    }
    int nhop = 0;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int n = n0 + k;
        if (n < n1) {
            if (lane < ZS) GX[gidx(n) * ZS + lane] = lane < MP ? x : S(0);
            x = hop_smem<S, MP>(pm[k], xb + ((nhop++) & 1) * RS, x, lane);
        }
    }
    if (!last) {
        // hand the state to the next warp (this warp's GX entries are read by
        // bulk copies once the last warp publishes)
        if (lane < RS) xh[warp * RS + lane] = lane < MP ? x : S(0);
        fence_proxy_async_global();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(hb + warp))
                                    : "memory");
        return true;
    }
    if (lane < ZS) GX[gidx(nh) * ZS + lane] = lane < MP ? x : S(0);
    fence_proxy_async_global();
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(cnt + b * kCntStride, 1u);
    return true;
}

// The body of k2_scan for block `bid` of `nblocks` (a mixed-order launch runs
// the bodies of several orders, each block one of them; every block of the
// launch is resident, so the waits between blocks of one order end).
template <typename S, int MP, int MODE, int DEPTH = kScanDepth>
__device__ __forceinline__ void scan_body(int64_t bid, int64_t nblocks, Batch bt, int M, int64_t items_bound,
                                          const S *__restrict__ Y, const S *__restrict__ Z, S *__restrict__ GY,
                                          S *__restrict__ GZ, S *__restrict__ GX, const S *__restrict__ zi,
                                          S *__restrict__ X, S *__restrict__ ckpt, unsigned *__restrict__ cnt,
                                          int *__restrict__ status, int *__restrict__ fix_list,
                                          int64_t n_chain = 0, int chain_regs = 0) {
    using SG = ScanGeo<S, MP, DEPTH>;
    constexpr int YS = SG::YS, ZS = SG::ZS, RS = SG::RS;
    constexpr bool REV = ScanMode<MODE>::REV;
    constexpr bool TRANS = ScanMode<MODE>::TRANS;
    constexpr bool VEC = ScanMode<MODE>::VEC;
    extern __shared__ __align__(128) unsigned char k2_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the last n_chain blocks of the launch run the chains (phase B1), one
    // signal at a time in warp 0; the others work on scan items
    if constexpr (DEPTH == kScanDepth) {
        if (bid >= nblocks - n_chain) {
            const int64_t cb = bid - (nblocks - n_chain);
            if constexpr (ChainRegs<S, MP>::ON) {
                // one signal per chain block, its chain short enough for the
                // warps' registers (it waits for the previous kernel itself)
                if (chain_regs && n_chain >= bt.n && cb < bt.n &&
                    sig_scan(bt, cb).nG - 1 <= kScanWarps * ChainRegs<S, MP>::KM) {
                    chain_block_regs<S, MP, MODE>(cb, bt, M, items_bound, GY, GZ, GX, zi, cnt, status);
                    return;
                }
            }
            pdl_wait();
            pdl_release();
            if (warp == 0) chain_block<S, MP, MODE>(cb, n_chain, bt, M, items_bound, GY, GZ, GX, zi, cnt, status);
            return;
        }
    }
    nblocks -= n_chain;
    const int64_t w0 = bid * kScanWarps + warp;
    const int64_t wstep = nblocks * kScanWarps;
    int64_t n_items = items_bound;
    if (bt.off != nullptr) {
        const int64_t n = __ldg(bt.gstart + bt.n);
        n_items = n < items_bound ? n : items_bound;
    }
    ScanWarp<S, MP, DEPTH> W;
    W.init(k2_smem + (size_t)warp * SG::WARP_BYTES, lane, status);
    S *xb = W.xb;
    const int j0 = lane < MP ? lane : 0;
    int nhop = 0;  // hops so far (selects the exchange buffer)

    // scan item -> (signal, group) and the signal's scan geometry
    // the batch's chunks (the chunk-map and list regions hold at least these)
    const int64_t total_chunks = bt.off == nullptr ? (int64_t)bt.n * bt.nC : (int64_t)__ldg(bt.cstart + bt.n);
    auto locate = [&](int64_t item, int64_t &b, int &g, SigScan &sg) {
        b = bt.off == nullptr ? item / bt.nG : (int64_t)find_signal(bt.gstart, bt.n, item);
        sg = sig_scan(bt, b);
        g = (int)(item - sg.gbase);
    };
    // a located item lies in its signal's groups, and the signal's chunks
    // and groups in the batch's (checked builds; skip the item otherwise)
    auto located_ok = [&](int64_t b, int g, const SigScan &sg) -> bool {
        return index_ok(b >= 0 && b < bt.n && g >= 0 && g < sg.nG && sg.gbase + sg.nG <= items_bound, CHK_SCAN_ITEM,
                        status) &&
               index_ok(sg.cbase >= 0 && sg.cbase + sg.nC <= total_chunks, CHK_SCAN_CHUNK, status);
    };
    auto group_len = [&](const SigScan &sg, int g) -> int {
        const int64_t lo = (int64_t)g * sg.G2;
        return (int)((lo + sg.G2 <= sg.nC ? lo + sg.G2 : sg.nC) - lo);
    };
    // chunk (within the signal) of the group's i-th step along the chain
    auto chunk_at = [&](const SigScan &sg, int g, int len, int i) -> int64_t {
        return (int64_t)g * sg.G2 + (REV ? len - 1 - i : i);
    };
    // the group's chunk maps (and z vectors), lowest address first
    auto group_maps = [&](const SigScan &sg, int g) -> const S * {
        return Y + (sg.cbase + (int64_t)g * sg.G2) * YS;
    };
    auto group_zs = [&](const SigScan &sg, int g) -> const S * {
        return VEC ? Z + (sg.cbase + (int64_t)g * sg.G2) * ZS : nullptr;
    };
    auto hop_step = [&](const S *m, const S *z, S x) -> S {
        S p[MP + 1];
        map_cols<S, MP, TRANS, VEC>(p, m, z, j0);
        return hop_smem<S, MP>(p, xb + ((nhop++) & 1) * RS, x, lane);
    };
    // the same hop, also giving the lane's component of P x (the map's
    // constant term taken off again)
    auto hop_step_pe = [&](const S *m, const S *z, S x, S &pe) -> S {
        S p[MP + 1];
        map_cols<S, MP, TRANS, VEC>(p, m, z, j0);
        const S xn = hop_smem<S, MP>(p, xb + ((nhop++) & 1) * RS, x, lane);
        pe = xn - p[0];
        return xn;
    };
    // bounded wait until signal b's counter reaches `target` (counted from
    // where the main scan left it, for a correction scan)
    auto wait_count = [&](int64_t b, const SigScan &sg, unsigned target) -> bool {
        const unsigned base = ScanMode<MODE>::FIX ? (unsigned)sg.nG + 1u : 0u;
        return wait_counter<64>(cnt + b * kCntStride, base + target, lane, status);
    };
    // make this warp's global stores visible (also to bulk copies) before
    // bumping signal b's counter
    auto publish = [&](int64_t b) {
        fence_proxy_async_global();
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(cnt + b * kCntStride, 1u);
    };

    // A vector scan's chunk maps come from a kernel two or more launches
    // back (the z vectors from the previous one): the copy of the first
    // group's maps into slots 0 .. len-1 starts before the wait.
    bool pre = false;
    if constexpr (VEC) {
        if (w0 < n_items) {
            int64_t b;
            int g;
            SigScan sg;
            locate(w0, b, g, sg);
            if (located_ok(b, g, sg) && group_len(sg, g) <= DEPTH) {
                W.issue(0, group_len(sg, g), group_maps(sg, g), nullptr, 0);
                pre = true;
            }
        }
    }
    pdl_wait();
    pdl_release();

    // ---- phase A: fold every group's chunk maps; the counter of signal b
    // reaches its group count when all its groups are done ----
    for (int64_t item = w0; item < n_items; item += wstep) {
        int64_t b;
        int g;
        SigScan sg;
        locate(item, b, g, sg);
        if (!located_ok(b, g, sg)) continue;
        const int len = group_len(sg, g);
        bool ok;
        if constexpr (VEC) {
            S zeta = S(0);
            if (pre && item == w0) {
                // the maps are on their way: add the z vectors
                W.issue_z(0, len, group_zs(sg, g), 1);
                const bool ok0 = W.wait(0), ok1 = W.wait(1);
                if (!ok0 || !ok1) {
                    if (!ok0) W.drain(0);
                    if (!ok1) W.drain(1);
                    return;
                }
                for (int i = 0; i < len; ++i) {
                    const int mi = REV ? len - 1 - i : i;
                    zeta = hop_step(W.map(mi), W.zv(mi), zeta);
                }
                ok = true;
            } else {
                ok = run_maps<S, MP, REV, DEPTH>(W, group_maps(sg, g), group_zs(sg, g), len,
                                                 [&](int, const S *m, const S *z) { zeta = hop_step(m, z, zeta); });
            }
            if (lane < ZS) GZ[item * ZS + lane] = lane < MP ? zeta : S(0);
        } else if constexpr (UseMma<S, MP>::ON) {
            // the running product in the warp's tile, starting from the
            // identity (y = 0); each map left-multiplies it on the tensor cores
            using MG = MmaGeo<MP>;
            float *rs = W.rs;
            for (int idx = lane; idx < MG::KP * MG::ST; idx += 32) {
                const int r = idx / MG::ST, j = idx - r * MG::ST;
                rs[idx] = (r == j && j < MP) ? 1.f : 0.f;
            }
            __syncwarp();
            ok = run_maps<S, MP, REV, DEPTH>(W, group_maps(sg, g), nullptr, len,
                                      [&](int, const S *m, const S *) { compose_mma<MP>(rs, m, lane); });
            // row 0 of the group map: y_g (column MP); row j+1: column j of Phi_g
            S *gy = GY + item * YS;
            for (int idx = lane; idx < (MP + 1) * RS; idx += 32) {
                const int r = idx / RS, k = idx - r * RS;
                gy[idx] = k < MP ? rs[k * MG::ST + (r == 0 ? MP : r - 1)] : S(0);
            }
        } else {
            // lane j < MP holds column j of the composed transfer (its response
            // to a unit incoming component j+1); the accumulated response y
            // rides on lane MP, or, for MP = 32, on a hop chain
            S col[MP];
#pragma unroll
            for (int k = 0; k < MP; ++k) col[k] = (k == lane) ? S(1) : S(0);
            S yv = S(0);
            ok = run_maps<S, MP, REV, DEPTH>(W, group_maps(sg, g), nullptr, len, [&](int, const S *m, const S *) {
                if constexpr (!YLane<MP>::ON) yv = hop_step(m, nullptr, yv);
                compose_step<S, MP>(col, m, lane);
            });
            S *gy = GY + item * YS;
            if constexpr (YLane<MP>::ON) {
                // lane j < MP: row j+1 (column j of Phi_g); lane MP: row 0 (y_g)
                if (lane <= MP) {
                    S *row = gy + (lane == MP ? 0 : (lane + 1) * RS);
#pragma unroll
                    for (int k = 0; k < RS; ++k) row[k] = k < MP ? col[k] : S(0);
                }
            } else {
                if (lane < RS) gy[lane] = lane < MP ? yv : S(0);
                if (lane < MP) {
                    S *row = gy + (lane + 1) * RS;
#pragma unroll
                    for (int k = 0; k < RS; ++k) row[k] = k < MP ? col[k] : S(0);
                }
            }
        }
        if (!ok) return;
        publish(b);
    }
    // With one item per warp whose group fits the buffers, they still hold
    // that group's chunk maps (memory order, slots 0 .. len-1).
    bool held = false;
    if (w0 < n_items && w0 + wstep >= n_items) {
        int64_t b;
        int g;
        SigScan sg;
        locate(w0, b, g, sg);
        held = located_ok(b, g, sg) && group_len(sg, g) <= DEPTH;
    }

    // ---- phase B1: the warp owning group 0 of a signal chains that
    // signal's group maps once, storing every group's incoming state in GX;
    // its count then reaches the group count + 1 ----
    for (int64_t item = w0; n_chain == 0 && item < n_items; item += wstep) {
        int64_t b;
        int g;
        SigScan sg;
        locate(item, b, g, sg);
        if (!located_ok(b, g, sg)) continue;
        if (g != 0) continue;
        held = false;
        const int nG = sg.nG;
        if (!wait_count(b, sg, (unsigned)nG)) return;
        fence_proxy_async_global();  // the group maps are read by bulk copies
        auto gidx = [&](int n) -> int64_t { return sg.gbase + (REV ? nG - 1 - n : n); };
        S x = S(0);
        if (MODE == CH_FWD && zi != nullptr) {
            const int64_t gs_ = global_signal(bt, b);
            const int m = bt.ord != nullptr ? __ldg(bt.ord + gs_) : M;
            if (lane < m) x = zi[gs_ * (bt.ldz > 0 ? bt.ldz : M) + lane];
        }
        // groups 0 .. nG-2 along the chain: the signal's group maps
        // [gbase, gbase + nG-1) forward, [gbase + 1, gbase + nG) backward
        const int64_t lo = sg.gbase + (REV ? 1 : 0);
        const bool ok = run_maps<S, MP, REV, DEPTH>(W, GY + lo * YS, VEC ? GZ + lo * ZS : nullptr, nG - 1,
                                             [&](int n, const S *m, const S *z) {
                                                 if (lane < ZS) GX[gidx(n) * ZS + lane] = lane < MP ? x : S(0);
                                                 x = hop_step(m, z, x);
                                             });
        if (!ok) return;
        if (lane < ZS) GX[gidx(nG - 1) * ZS + lane] = lane < MP ? x : S(0);
        publish(b);
    }

    // ---- phase B2: every group runs its chunks from its incoming state,
    // writing each chunk's incoming state X (and the forward's checkpoints) ----
    for (int64_t item = w0; item < n_items; item += wstep) {
        int64_t b;
        int g;
        SigScan sg;
        locate(item, b, g, sg);
        if (!located_ok(b, g, sg)) continue;
        const int len = group_len(sg, g);
        if (!wait_count(b, sg, (unsigned)sg.nG + 1u)) return;
        constexpr bool FIX = ScanMode<MODE>::FIX;
        const float fix_bar = FIX ? kFixTheta * scale_of(cnt, b) : 0.f;
        // pe (FIX): the lane's component of P_c x, the chunk's correction
        // carried to the chunk's end
        auto put = [&](int ci, S x, S pe) {
            const int64_t q = sg.cbase + chunk_at(sg, g, len, ci);
            if (lane < MP) X[q * MP + lane] = x;
            if (MODE == CH_FWD && ckpt != nullptr && lane < M) ckpt[q * M + lane] = x;
            if constexpr (FIX) {
                // list the chunk for pass 2 when its correction, at its start
                // or carried to its end, is finite and above the threshold
                // of its (finite) signal
                // one warp max over the bit patterns: for non-negative
                // floats they order as the values, and a NaN (sign cleared)
                // stays above every finite value and infinity
                const float el = lane < MP ? fabsf((float)abs_max_nan(fabs(x), pe)) : 0.f;
                const float em = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(el)));
                if (lane == 0 && em > fix_bar && em <= 3.0e38f) {
                    const unsigned slot = atomicAdd(cnt + (int64_t)bt.n * kCntStride, 1u);
                    if (index_ok((int64_t)slot < total_chunks, CHK_FIX_LIST_SLOT, status)) fix_list[slot] = (int)q;
                }
            }
        };
        S x = lane < MP ? __ldcg(GX + item * ZS + lane) : S(0);
        auto step = [&](int i, const S *m, const S *z) {
            if constexpr (FIX) {
                S pe;
                const S xn = hop_step_pe(m, z, x, pe);
                put(i, x, pe);
                x = xn;
            } else {
                put(i, x, S(0));
                x = hop_step(m, z, x);
            }
        };
        // the main scans need every map of the group but the last along the
        // chain; the correction scans also carry the last chunk's correction
        // through its own map
        const int nh = FIX ? len : len - 1;
        if (held) {
            // the group's maps are still in slots 0 .. len-1
            for (int i = 0; i < nh; ++i) {
                const int mi = REV ? len - 1 - i : i;
                step(i, W.map(mi), W.zv(mi));
            }
        } else {
            const int64_t off = (REV && !FIX) ? 1 : 0;
            const S *zlo = VEC ? group_zs(sg, g) + off * ZS : nullptr;
            if (!run_maps<S, MP, REV, DEPTH>(W, group_maps(sg, g) + off * YS, zlo, nh, step)) return;
        }
        if (!FIX) put(len - 1, x, S(0));
    }
}

// With the register chain compiled in, one block per SM as the launch bound
// lets ptxas give every variant its registers without spilling (shared
// memory holds the scan to two blocks per SM in any case).
template <typename S, int MP, int MODE>
__global__ void __launch_bounds__(kScanWarps * 32, ChainRegs<S, MP>::ON ? 1 : 0)
    k2_scan(Batch bt, int M, int64_t items_bound, const S *__restrict__ Y, const S *__restrict__ Z,
            S *__restrict__ GY, S *__restrict__ GZ, S *__restrict__ GX, const S *__restrict__ zi,
            S *__restrict__ X, S *__restrict__ ckpt, unsigned *__restrict__ cnt, int *__restrict__ status,
            int *__restrict__ fix_list, int n_chain, int chain_regs) {
    scan_body<S, MP, MODE>(blockIdx.x, gridDim.x, bt, M, items_bound, Y, Z, GY, GZ, GX, zi, X, ckpt, cnt, status,
                           fix_list, n_chain, chain_regs);
}

// ---------------------------------------------------------------------------
// Coefficient gradient (Eq. 12): ga[b][t][i-1] = -ge(b,t) * s(b, t-i), with
// s(b, -j) = zi[b][j-1] (zero without zi).  A block owns TR rows of one
// signal: it stages the s window in shared memory, builds its TR*M outputs
// (one contiguous span) in a shared tile, one row per thread, and writes
// the span with one bulk copy when it is 16-byte aligned.
// ---------------------------------------------------------------------------
template <typename S, int MP, bool EXACT> struct GradGeo {
    static constexpr int TR = 256;       // rows per block
    static constexpr int THREADS = 256;
};

// largest b in [0, n) with off[b] <= t (off non-decreasing, off[0] = 0)
__device__ __forceinline__ int find_row_signal(const int64_t *__restrict__ off, int n, int64_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename S, int MP, bool EXACT>
__global__ void __launch_bounds__(256)
    k_grad_a(Batch bt, int M, int64_t tiles_per_signal, const S *__restrict__ ge, const S *__restrict__ s,
             const S *__restrict__ zi, S *__restrict__ ga) {
    constexpr int TR = GradGeo<S, MP, EXACT>::TR;
    __shared__ S s_t[TR + MP];
    const bool varlen = bt.off != nullptr;
    // uniform: the block owns rows [t0, t0+TR) of signal b, row r at b*T + t;
    // varlen: the block owns packed rows [t0, t0+TR), each in its own signal
    int64_t b = 0, t0, row0, nrows;
    if (varlen) {
        t0 = (int64_t)blockIdx.x * TR;
        row0 = t0;
        nrows = __ldg(bt.off + bt.n);
    } else {
        b = blockIdx.x / tiles_per_signal;
        t0 = (blockIdx.x - b * tiles_per_signal) * (int64_t)TR;
        row0 = b * bt.T + t0;
        nrows = bt.T;
    }
    if (t0 >= nrows) return;
    const int rows = (nrows - t0) < TR ? (int)(nrows - t0) : TR;
    for (int i = threadIdx.x; i < TR + MP; i += blockDim.x) {
        const int64_t t = t0 - MP + i;  // s_t[i] = s(t0 - MP + i), in the signal's rows (packed rows for varlen)
        S v = S(0);
        if (t >= 0 && t < nrows) v = s[row0 - t0 + t];
        else if (!varlen && t < 0 && zi != nullptr && -t <= M) v = zi[b * M + (-t - 1)];
        s_t[i] = v;
    }
    // s comes from the forward, two or more launches back; ge from the
    // kernel just before this one
    pdl_wait();
    pdl_release();
    // varlen: history before a row's own signal start is that signal's zi
    auto hist = [&](int r, int i, int64_t rb, int64_t ro) -> S {
        const int64_t tt = t0 + r - 1 - i;
        if (!varlen || tt >= ro) return s_t[MP + r - 1 - i];
        const int64_t j = ro - tt;  // s_b(-j) = zi[b][j-1]
        return (zi != nullptr && j <= M) ? zi[rb * M + (j - 1)] : S(0);
    };
    if constexpr (EXACT) {
        // thread r computes row t0+r into a shared tile laid out like the
        // output; the block's rows*MP outputs then leave as one bulk copy
        __shared__ __align__(128) S tile[TR * MP];
        const int r = threadIdx.x;
        const S g = r < rows ? ge[row0 + r] : S(0);
        __syncthreads();
        if (r < rows) {
            if (varlen) {
                const int64_t rb = find_row_signal(bt.off, bt.n, t0 + r), ro = __ldg(bt.off + rb);
#pragma unroll
                for (int i = 0; i < MP; ++i) tile[r * MP + i] = -g * hist(r, i, rb, ro);
            } else {
#pragma unroll
                for (int i = 0; i < MP; ++i) tile[r * MP + i] = -g * s_t[MP + r - 1 - i];
            }
        }
        fence_proxy_async();
        __syncthreads();
        S *dst = ga + row0 * (int64_t)MP;
        const unsigned bytes = (unsigned)(rows * MP * sizeof(S));
        if (aligned16(dst) && bytes % 16 == 0) {
            if (threadIdx.x == 0) {
                bulk_store(dst, tile, bytes);
                bulk_store_commit_wait();
            }
        } else {
            for (int idx = threadIdx.x; idx < rows * MP; idx += blockDim.x) dst[idx] = tile[idx];
        }
    } else {
        __shared__ S g_t[TR];
        __shared__ int64_t sig_t[TR], org_t[TR];
        for (int i = threadIdx.x; i < TR; i += blockDim.x) {
            g_t[i] = (i < rows) ? ge[row0 + i] : S(0);
            if (varlen && i < rows) {
                sig_t[i] = find_row_signal(bt.off, bt.n, t0 + i);
                org_t[i] = __ldg(bt.off + sig_t[i]);
            }
        }
        __syncthreads();
        S *dst = ga + row0 * (int64_t)M;
        for (int idx = threadIdx.x; idx < rows * M; idx += blockDim.x) {
            const int rr = idx / M, i = idx - rr * M;  // i = coefficient index - 1
            dst[idx] = -g_t[rr] * (varlen ? hist(rr, i, sig_t[rr], org_t[rr]) : s_t[MP + rr - (i + 1)]);
        }
    }
}

// ---------------------------------------------------------------------------
// Gradients with respect to generated coefficients (uniform batches, FP32).
// Both start from Eq. 12, dL/da_i(t) = -ge(t) s(t-i) with s(t-i) = zi[i-t-1]
// for t < i, and never store it.
// ---------------------------------------------------------------------------
constexpr int kGradRows = 1024;  // rows of one time-invariant gradient tile
constexpr int kGradThreads = 128;

// SRC_CONST (Eq. 3: the time-invariant gradient is Eq. 12 summed over time):
// part[b][tile][i] = sum over the tile's rows t of ge(t) s(t-i-1) (the sign
// is applied by k_grad_finish).  Threads (grp, i): grp = tid / 32 takes rows
// grp, grp + 4, ... of the tile; the four groups are added in a fixed order.
template <int MP>
__global__ void __launch_bounds__(kGradThreads)
    k_grad_const(int64_t T, int M, int64_t tiles, const float *__restrict__ ge, const float *__restrict__ s,
                 const float *__restrict__ zi, float *__restrict__ part) {
    __shared__ float sg[kGradRows];
    __shared__ float ss[kGradRows + MP];
    __shared__ float red[kGradThreads / 32][32];
    const int64_t b = blockIdx.y, tile = blockIdx.x;
    const int64_t t0 = tile * kGradRows;
    const int tid = threadIdx.x;
    pdl_wait();
    pdl_release();
    for (int r = tid; r < kGradRows + MP; r += kGradThreads) {
        const int64_t t = t0 - MP + r;  // ss[r] = s(t0 - MP + r)
        float v = 0.f;
        if (t >= 0 && t < T) v = s[b * T + t];
        else if (t < 0 && zi != nullptr && -t <= M) v = zi[b * M + (-t - 1)];
        ss[r] = v;
        if (r < kGradRows) sg[r] = (t0 + r < T) ? ge[b * T + t0 + r] : 0.f;
    }
    __syncthreads();
    const int grp = tid / 32, i = tid % 32;
    float acc = 0.f;
    if (i < MP) {
        for (int r = grp; r < kGradRows; r += kGradThreads / 32) acc = fmaf(sg[r], ss[MP + r - i - 1], acc);
    }
    red[grp][i] = acc;
    __syncthreads();
    if (tid < MP) {
        float v = 0.f;
#pragma unroll
        for (int g = 0; g < kGradThreads / 32; ++g) v += red[g][tid];
        part[(b * tiles + tile) * MP + tid] = v;
    }
}

// gk[b][i] = -sum over tiles of part[b][tile][i], tiles in order.
static __global__ void k_grad_const_finish(int B, int M, int MP, int64_t tiles, const float *__restrict__ part,
                                    float *__restrict__ gk) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    pdl_wait();
    pdl_release();
    if (idx >= (int64_t)B * M) return;
    const int64_t b = idx / M;
    const int i = (int)(idx % M);
    float v = 0.f;
    for (int64_t t = 0; t < tiles; ++t) v += part[(b * tiles + t) * MP + i];
    gk[idx] = -v;
}

// SRC_FRAMES: one warp per (signal, frame segment f), samples
// t in [f hop, min((f+1) hop, T)).  Per sample, with G = dL/da(t):
//   step-up reversed (m = M .. 1), with A^(m) the order-m coefficients:
//     dL/dk_m(t) = G^(m)_m + sum_{i<m} G^(m)_i A^(m-1)_{m-i}
//     G^(m-1)_j  = G^(m)_j + k_m G^(m)_{m-j}            (j < m)
//   interpolation reversed: frame f gets (1 - w) dL/dk(t), frame f+1 gets
//   w dL/dk(t).
// A^(m) for the reverse sweep: the forward step-up keeps A at every SEG-th
// order, and each segment of orders is recomputed from its checkpoint, so
// everything stays in registers with compile-time indices.  The 32 lanes'
// dL/dk(t) go through shared memory and are summed per coefficient in a
// fixed order.  lo[b][f] and hi[b][f+1] receive the segment's two parts.
template <int MP> struct FrameGradGeo {
    static constexpr int SEG = 6;
    static constexpr int NSEG = (MP + SEG - 1) / SEG;
    static constexpr int WARPS = 4;
};

template <int MP>
__device__ __forceinline__ void stepup_stage(float (&a)[MP], float km, int m) {
    // m is a compile-time constant after unrolling
#pragma unroll
    for (int i = 1; 2 * i < MP + 1; ++i) {
        if (2 * i < m) {
            const float lo = a[i - 1], hi = a[m - i - 1];
            a[i - 1] = fmaf(km, hi, lo);
            a[m - i - 1] = fmaf(km, lo, hi);
        }
    }
    if (m % 2 == 0) a[m / 2 - 1] = fmaf(km, a[m / 2 - 1], a[m / 2 - 1]);
    a[m - 1] = km;
}

// Varlen batches (off != nullptr): items are the rows of the packed frame
// array k [n_frames][M]; signal b owns rows [foff[b], foff[b+1]) (the last
// up to n_frames) and samples [off[b], off[b+1]) of ge and s.
__device__ __forceinline__ int find_frame_signal(const int64_t *__restrict__ foff, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(foff + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int MP>
__global__ void __launch_bounds__(32 * FrameGradGeo<MP>::WARPS)
    k_grad_frames(int B, int64_t T, int M, int64_t F, int hop, float inv_hop, const float *__restrict__ k,
                  const float *__restrict__ ge, const float *__restrict__ s, const float *__restrict__ zi,
                  float *__restrict__ lo_out, float *__restrict__ hi_out, const int64_t *__restrict__ off,
                  const int64_t *__restrict__ foff) {
    using FG = FrameGradGeo<MP>;
    constexpr int SEG = FG::SEG, NSEG = FG::NSEG;
    __shared__ float gsh[FG::WARPS][32][MP + 1];
    __shared__ float wsh[FG::WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // uniform: item = b F + f, F frames per signal; varlen: F is the total
    // frame count and item a row of the packed frames
    const int64_t item = (int64_t)blockIdx.x * FG::WARPS + warp;
    pdl_wait();
    pdl_release();
    const int64_t n_items = off != nullptr ? F : (int64_t)B * F;
    if (item >= n_items) return;
    int64_t b, f, Fb, r0;  // signal, frame within it, its frames, its first row
    int64_t Tb;             // its samples
    if (off == nullptr) {
        b = item / F;
        f = item % F;
        Fb = F;
        r0 = b * T;
        Tb = T;
    } else {
        b = find_frame_signal(foff, B, item);
        const int64_t fb0 = __ldg(foff + b);
        f = item - fb0;
        Fb = (b + 1 < B ? __ldg(foff + b + 1) : F) - fb0;
        r0 = __ldg(off + b);
        Tb = __ldg(off + b + 1) - r0;
    }
    const int64_t ts = f * hop, te = ts + hop < Tb ? ts + hop : Tb;
    const float *k0 = k + item * (int64_t)M;
    const float *k1 = f + 1 < Fb ? k0 + M : k0;
    float lo_acc = 0.f, hi_acc = 0.f;  // lane m < M: coefficient m+1
    for (int64_t base = ts; base < te; base += 32) {
        const int64_t t = base + lane;
        const bool valid = t < te;
        float g[MP];  // G^(m) for the current m, g[i-1] = G_i
        float w = 0.f;
        if (valid) {
            w = (float)(t - ts) * inv_hop;
            const float gt = ge[r0 + t];
#pragma unroll
            for (int i = 1; i <= MP; ++i) {
                float sv = 0.f;
                if (i <= M) {
                    const int64_t u = t - i;
                    if (u >= 0) sv = s[r0 + u];
                    else if (zi != nullptr) sv = zi[b * M + (-u - 1)];
                }
                g[i - 1] = -gt * sv;
            }
        } else {
#pragma unroll
            for (int i = 0; i < MP; ++i) g[i] = 0.f;
        }
        // k(t) and the forward step-up with checkpoints every SEG orders
        float kt[MP];
#pragma unroll
        for (int m = 1; m <= MP; ++m) {
            float km = 0.f;
            if (m <= M) {
                const float x0 = __ldg(k0 + m - 1), x1 = __ldg(k1 + m - 1);
                km = fmaf(w, x1 - x0, x0);
            }
            kt[m - 1] = km;
        }
        float ck[NSEG][MP];
        {
            float a[MP];
#pragma unroll
            for (int i = 0; i < MP; ++i) a[i] = 0.f;
#pragma unroll
            for (int m = 1; m <= MP; ++m) {
                if (m % SEG == 1) {
#pragma unroll
                    for (int i = 0; i < MP; ++i) ck[(m - 1) / SEG][i] = a[i];  // A^(m-1)
                }
                stepup_stage<MP>(a, kt[m - 1], m);
            }
        }
        // dL/dk_m(t) goes straight to the warp's row of shared memory
        float *gk = gsh[warp][lane];
#pragma unroll
        for (int j = NSEG - 1; j >= 0; --j) {
            const int mlo = j * SEG;  // segment orders mlo+1 .. mhi
            const int mhi = (j + 1) * SEG < MP ? (j + 1) * SEG : MP;
            // A^(mlo) .. A^(mhi-1)
            float seg[SEG][MP];
#pragma unroll
            for (int i = 0; i < MP; ++i) seg[0][i] = ck[j][i];
#pragma unroll
            for (int q = 1; q < SEG; ++q) {
                if (mlo + q < mhi) {
#pragma unroll
                    for (int i = 0; i < MP; ++i) seg[q][i] = seg[q - 1][i];
                    stepup_stage<MP>(seg[q], kt[mlo + q - 1], mlo + q);
                }
            }
#pragma unroll
            for (int q = SEG - 1; q >= 0; --q) {
                const int m = mlo + q + 1;  // stage m uses A^(m-1) = seg[q]
                if (m <= mhi) {
                    float d = g[m - 1];
#pragma unroll
                    for (int i = 1; i < MP; ++i)
                        if (i < m) d = fmaf(g[i - 1], seg[q][m - i - 1], d);
                    gk[m - 1] = valid ? d : 0.f;
                    const float km = kt[m - 1];
#pragma unroll
                    for (int jj = 1; 2 * jj < MP + 1; ++jj) {
                        if (2 * jj < m) {
                            const float x = g[jj - 1], y = g[m - jj - 1];
                            g[jj - 1] = fmaf(km, y, x);
                            g[m - jj - 1] = fmaf(km, x, y);
                        }
                    }
                    if (m % 2 == 0) g[m / 2 - 1] = fmaf(km, g[m / 2 - 1], g[m / 2 - 1]);
                }
            }
        }
        wsh[warp][lane] = valid ? w : 0.f;
        __syncwarp();
        if (lane < MP) {
            float l = 0.f, h = 0.f;
            for (int r = 0; r < 32; ++r) {
                const float v = gsh[warp][r][lane], wr = wsh[warp][r];
                h = fmaf(wr, v, h);
                l = fmaf(1.f - wr, v, l);
            }
            lo_acc += l;
            hi_acc += h;
        }
        __syncwarp();
    }
    if (lane < M) {
        lo_out[item * (int64_t)M + lane] = lo_acc;
        if (f + 1 < Fb) hi_out[(item + 1) * (int64_t)M + lane] = hi_acc;
        if (f == 0) hi_out[item * (int64_t)M + lane] = 0.f;
    }
}

// gk = lo + hi, element by element.
static __global__ void k_grad_frames_finish(int64_t n, const float *__restrict__ lo, const float *__restrict__ hi,
                                     float *__restrict__ gk) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    pdl_wait();
    pdl_release();
    if (i < n) gk[i] = lo[i] + hi[i];
}

}  // namespace tvlp
