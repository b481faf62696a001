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
//   k2_group/chain/expand
//                   x_{c+1} = P_c x_c + y_c (forward) or
//                   w_{c-1} = P_c^T w_c + z_c (adjoint) per signal, as a
//                   two-level scan over groups of chunks.
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

namespace tvlp {

constexpr int SR = 8;    // rows per compute block (register window)
constexpr int SRS = 16;  // rows per staged copy; chunk lengths are multiples of SRS

// Status codes written by kernels to the device status word.
enum { DEV_OK = 0, DEV_TIMEOUT_TMA = 1 };

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
    static constexpr int UPL = (U_STAGE + 31) / 32;         // input samples each lane stages
    // per-warp slice: the stage ring then NS mbarriers, rounded to 128 bytes
    // so every warp's bulk-copy destinations stay 16-byte aligned
    static constexpr size_t RING_BYTES = size_t(NS) * (A_STAGE + U_STAGE) * sizeof(S);
    static constexpr size_t WARP_BYTES = ((RING_BYTES + NS * 8 + 127) / 128) * 128;
    static_assert(G * R >= MP + 1, "packing must hold MP+1 recursions");
    static_assert((CS * sizeof(S)) % 16 == 0, "16-byte stage alignment");
    static_assert((A_STAGE * sizeof(S)) % 16 == 0 && (U_STAGE * sizeof(S)) % 16 == 0, "16-byte ring alignment");
    static_assert(RING_BYTES % 8 == 0 && WARP_BYTES % 16 == 0, "mbarrier and warp-slice alignment");
};
// per-chunk stride of the summaries Y[c][MP+1][MP], a multiple of 16 bytes
template <typename S, int MP> struct YGeo {
    static constexpr int YS = (((MP + 1) * MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
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

constexpr int kWaitLimit = 1 << 22;  // mbarrier polls before a wait gives up

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
// K1: chunk summaries.
// Flattened chunk index q = b*nC + c; chunk c of signal b covers samples
// [c*L, c*L + L).  Each warp owns CPW consecutive chunks; lane (grp = lane/G,
// g = lane%G) runs recursions r = g*R + k, k < R.  Coefficient rows are
// staged in shared memory, SRS rows per stage, two stages in a ring: a full,
// 16-byte-aligned chunk-stage arrives as one bulk (TMA) copy completing on
// the stage's mbarrier; others (a ragged tail, a misaligned start, a padded
// order) use cp.async with zero fill.  Input samples are loaded by the warp
// one stage ahead and parked in shared memory next to the coefficients.
// Output Y[q][r][k] (per-chunk stride YS):
//   forward:  s(c*L + L - 1 - k) of recursion r
//   backward: q_{k+1} after the chunk, i.e. the pending dL/ds(c*L - 1 - k)
// ---------------------------------------------------------------------------
template <typename S, int MP, typename GE, bool BWD>
__device__ __forceinline__ void k1_issue_stage(S *a_st, uint64_t *bar, const S *__restrict__ a, int M, int L, int k,
                                               int lane, int64_t my_base, int my_valid, bool exact) {
    constexpr int CPW = GE::CPW;
    constexpr unsigned A_BYTES = SRS * MP * sizeof(S);
    const int roff = BWD ? L - (k + 1) * SRS : k * SRS;  // chunk-local first row of the stage
    int nvalid = my_valid - roff;
    nvalid = nvalid < 0 ? 0 : (nvalid > SRS ? SRS : nvalid);
    const bool mine = lane < CPW;
    const S *src_a = a + (my_base + roff) * (int64_t)MP;
    const bool tma_a = mine && exact && nvalid == SRS && aligned16(src_a);
    const unsigned ntma = __popc(__ballot_sync(0xffffffffu, tma_a));
    if (lane == 0) mbar_arrive_expect_tx(bar, ntma * A_BYTES);
    __syncwarp();
    if (tma_a) {
        fence_proxy_async();
        bulk_load(a_st + lane * GE::CS, src_a, A_BYTES, bar);
    }
    // fallback chunk-stages
    unsigned slow = __ballot_sync(0xffffffffu, mine && !tma_a);
    while (slow) {
        const int ch = __ffs(slow) - 1;
        slow &= slow - 1;
        const int64_t base = __shfl_sync(0xffffffffu, my_base, ch);
        const int nv = __shfl_sync(0xffffffffu, nvalid, ch);
        S *dst = a_st + ch * GE::CS;
        if (exact) {
            const S *s0 = a + (base + roff) * (int64_t)MP;
            for (int idx = lane; idx < SRS * MP; idx += 32) {
                const bool v = idx < nv * MP;
                cp_async<sizeof(S)>(dst + idx, v ? s0 + idx : a, v ? (int)sizeof(S) : 0);
            }
        } else {
            // padded order: the M real coefficients of every row; the padded
            // columns were zeroed once and are never written
            for (int r = 0; r < SRS; ++r) {
                if (lane < M) {
                    const bool v = r < nv;
                    const S *s0 = v ? a + (base + roff + r) * (int64_t)M + lane : a;
                    cp_async<sizeof(S)>(dst + r * MP + lane, s0, v ? (int)sizeof(S) : 0);
                }
            }
        }
    }
    cp_async_commit();
}

// Input samples of stage k for the warp's chunks: element e = lane + 32*i
// (i < UPL) is row e % SRS of chunk e / SRS; zero past the signal's end.
template <typename S, int MP, typename GE, bool BWD>
__device__ __forceinline__ void k1_load_inputs(S (&uv)[GE::UPL], const S *__restrict__ u, int L, int k, int lane,
                                               int64_t my_base, int my_valid) {
    const int roff = BWD ? L - (k + 1) * SRS : k * SRS;
#pragma unroll
    for (int i = 0; i < GE::UPL; ++i) {
        const int e = lane + 32 * i;
        const int ch = (e / SRS) < GE::CPW ? e / SRS : 0;
        const int64_t base = __shfl_sync(0xffffffffu, my_base, ch);
        const int valid = __shfl_sync(0xffffffffu, my_valid, ch);
        const int r = e % SRS;
        uv[i] = (e < GE::U_STAGE && roff + r < valid) ? __ldg(u + base + roff + r) : S(0);
    }
}

template <typename S, int MP, int G, int R, bool BWD>
__global__ void __launch_bounds__(256, 1)
    k1_summary(int64_t T, int M, int L, int64_t nC, int64_t NQ, const S *__restrict__ a, const S *__restrict__ u,
               S *__restrict__ Y, int exact_flag, int *__restrict__ status) {
    using GE = SumGeo<S, MP, G, R>;
    constexpr int CPW = GE::CPW, NS = GE::NS, WIN = MP + SR;
    constexpr int YS = YGeo<S, MP>::YS;
    extern __shared__ __align__(128) unsigned char k1_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t q0 = ((int64_t)blockIdx.x * wpb + warp) * CPW;
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
    // lane ch < CPW describes chunk q0 + ch: first row b*T + c*L, valid rows
    int64_t my_base = 0;
    int my_valid = 0;
    if (lane < CPW && q0 + lane < NQ) {
        const int64_t q = q0 + lane;
        const int64_t b = q / nC;
        const int64_t t0 = (q - b * nC) * (int64_t)L;
        my_base = b * T + t0;
        const int64_t rem = T - t0;
        my_valid = rem < L ? (int)rem : L;
    }
    const int grp = lane / G, g = lane % G;
    const int nblk = L / SRS;

    // forward window: h[k][MP - i] = s(t - i) at a block start; backward
    // window: h[k][j - 1] = q_j at a block start
    S h[R][WIN];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = g * R + k;
#pragma unroll
        for (int m = 0; m < WIN; ++m) {
            const int unit = BWD ? r - 1 : MP - r;
            h[k][m] = (r >= 1 && r <= MP && m == unit) ? S(1) : S(0);
        }
    }
    const S flag0 = (g == 0) ? S(1) : S(0);

    S uv[GE::UPL];
    k1_issue_stage<S, MP, GE, BWD>(a_buf, bars, a, M, L, 0, lane, my_base, my_valid, exact);
    k1_load_inputs<S, MP, GE, BWD>(uv, u, L, 0, lane, my_base, my_valid);
#pragma unroll
    for (int i = 0; i < GE::UPL; ++i)
        if (lane + 32 * i < GE::U_STAGE) u_buf[lane + 32 * i] = uv[i];
#pragma unroll 1
    for (int k = 0; k < nblk; ++k) {
        const int slot = k & 1;
        const bool more = k + 1 < nblk;
        if (more) {
            // the other slot was consumed in the previous iteration
            k1_issue_stage<S, MP, GE, BWD>(a_buf + (slot ^ 1) * GE::A_STAGE, bars + (slot ^ 1), a, M, L, k + 1, lane,
                                           my_base, my_valid, exact);
            k1_load_inputs<S, MP, GE, BWD>(uv, u, L, k + 1, lane, my_base, my_valid);
        } else {
            cp_async_commit();
        }
        cp_async_wait<1>();
        if (!mbar_wait_warp(bars + slot, (k >> 1) & 1, kWaitLimit)) {
            // a bulk copy never completed: record it, give the copy this warp
            // still has in flight a bounded chance to land, and leave
            if (lane == 0) atomicExch(status, DEV_TIMEOUT_TMA);
            if (more) mbar_wait_warp(bars + (slot ^ 1), ((k + 1) >> 1) & 1, kWaitLimit);
            cp_async_wait<0>();
            return;
        }
        __syncwarp();
        const S *arow = a_buf + slot * GE::A_STAGE + grp * GE::CS;
        const S *urow = u_buf + slot * GE::U_STAGE + grp * SRS;
#pragma unroll
        for (int cb = 0; cb < SRS / SR; ++cb) {
            // forward: rows cb*SR + j; backward: the stage's rows in reverse
            const int rb = BWD ? (SRS / SR - 1 - cb) * SR : cb * SR;
#pragma unroll
            for (int j = 0; j < SR; ++j) {
                const int row = BWD ? rb + SR - 1 - j : rb + j;
                S c[MP];
                load_row_smem<S, MP>(c, arow + row * MP);
                const S uu = flag0 * urow[row];
                if constexpr (BWD) {
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
#pragma unroll
            for (int kk = 0; kk < R; ++kk) slide<S, MP, WIN>(h[kk]);
        }
        // park the next stage's input samples in the slot this iteration read
        // last time round (consumed before the previous iteration ended)
        if (more) {
#pragma unroll
            for (int i = 0; i < GE::UPL; ++i)
                if (lane + 32 * i < GE::U_STAGE) u_buf[(slot ^ 1) * GE::U_STAGE + lane + 32 * i] = uv[i];
        }
        __syncwarp();
    }
    // end states
    const int64_t q = q0 + grp;
    if (q < NQ) {
        S *yq = Y + q * YS;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int r = g * R + k;
            if (r <= MP) {
#pragma unroll
                for (int j = 0; j < MP; ++j) yq[r * MP + j] = BWD ? h[k][j] : h[k][MP - 1 - j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// One recursion per lane over its chunk ("lane per chunk"): a warp owns 32
// consecutive chunks.  Each lane has a private ring of two stages of SRS
// coefficient rows; a full, aligned lane-stage arrives by one bulk copy
// completing on the warp's per-stage mbarrier, others by cp.async with zero
// fill.  Input samples are loaded into registers one stage ahead.
//   FWD_RERUN: start from X[q] (or zi / zero), write s.
//   BWD_ZERO:  adjoint from zero state, store the end state to Z[q].
//   BWD_RERUN: adjoint from W[q], write ge; chunk 0 also writes gzi.
// A launch with one chunk per signal (L >= T) is the plain sequential filter.
// With `reverse` set, warps walk the chunks from the end, so a pass right
// after another over the same rows starts with the rows that pass loaded
// last (most likely still in L2).
// ---------------------------------------------------------------------------
enum { FWD_RERUN = 0, BWD_ZERO = 1, BWD_RERUN = 2 };

template <typename S, int MP> struct RecGeo {
    static constexpr int NS = 2;                                    // stages per lane ring
    static constexpr int A_ST = SRS * MP;                           // coefficient elements per lane-stage
    static constexpr int RAW = (NS * A_ST * (int)sizeof(S)) / 4;    // words per lane
    // lane stride in words: an odd multiple of 4, so the 16-byte row loads of
    // a quarter warp hit distinct bank quads
    static constexpr int LW = ((RAW + 3) / 4) % 2 == 1 ? ((RAW + 3) / 4) * 4 : ((RAW + 3) / 4 + 1) * 4;
    static constexpr size_t SMEM = size_t(32) * LW * 4 + NS * 8;
    static_assert((A_ST * sizeof(S)) % 16 == 0, "16-byte lane stages");
    static_assert((LW * 4) % 16 == 0, "16-byte lane ring alignment");
    static_assert(NS * A_ST * sizeof(S) <= size_t(LW) * 4, "lane ring fits its stride");
};

template <typename S, int MP, bool EXACT, bool BWD>
__device__ __forceinline__ void rec_issue_stage(S *a_st, uint64_t *bar, const S *__restrict__ a, int M, int L, int s,
                                                bool active, int64_t base, int n) {
    constexpr unsigned A_BYTES = SRS * MP * sizeof(S);
    const int roff = BWD ? L - (s + 1) * SRS : s * SRS;
    int nv = n - roff;
    nv = nv < 0 ? 0 : (nv > SRS ? SRS : nv);
    if (!active) nv = 0;
    const S *src_a = a + (base + roff) * (int64_t)M;
    const bool tma_a = EXACT && nv == SRS && aligned16(src_a);
    const unsigned ntma = __popc(__ballot_sync(0xffffffffu, tma_a));
    if ((threadIdx.x & 31) == 0) mbar_arrive_expect_tx(bar, ntma * A_BYTES);
    __syncwarp();
    if (tma_a) {
        fence_proxy_async();
        bulk_load(a_st, src_a, A_BYTES, bar);
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

template <typename S, bool BWD>
__device__ __forceinline__ void rec_load_inputs(S (&uv)[SRS], const S *__restrict__ u, int L, int s, bool active,
                                                int64_t base, int n) {
    const int roff = BWD ? L - (s + 1) * SRS : s * SRS;
#pragma unroll
    for (int r = 0; r < SRS; ++r) uv[r] = (active && roff + r < n) ? __ldg(u + base + roff + r) : S(0);
}

template <typename S, int MP, bool EXACT, int MODE>
__global__ void __launch_bounds__(32)
    k_rec(int64_t T, int M, int L, int64_t nC, int64_t NQ, const S *__restrict__ a, const S *__restrict__ u,
          const S *__restrict__ Xin, const S *__restrict__ zi, S *__restrict__ out, S *__restrict__ Zout,
          S *__restrict__ gzi, int reverse, int *__restrict__ status) {
    using RG = RecGeo<S, MP>;
    constexpr int NS = RG::NS, WIN = MP + SR;
    constexpr bool BWD = MODE != FWD_RERUN;
    extern __shared__ __align__(128) unsigned char rec_smem[];
    const int lane = threadIdx.x & 31;
    const int64_t blk = reverse ? (int64_t)gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int64_t q = blk * 32 + lane;
    const bool active = q < NQ;
    S *a_ring = reinterpret_cast<S *>(rec_smem + (size_t)lane * RG::LW * 4);  // [NS][SRS*MP]
    uint64_t *bars = reinterpret_cast<uint64_t *>(rec_smem + (size_t)32 * RG::LW * 4);
    if (!EXACT) {
        for (int j = 0; j < NS * RG::A_ST; ++j) a_ring[j] = S(0);
    }
    if (lane == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    int64_t b = 0, c = 0, base = 0;
    int n = 0;
    if (active) {
        b = q / nC;
        c = q - b * nC;
        const int64_t t0 = c * (int64_t)L;
        base = b * T + t0;
        const int64_t rem = T - t0;
        n = rem < L ? (int)rem : L;
    }
    S h[WIN];
#pragma unroll
    for (int m = 0; m < WIN; ++m) h[m] = S(0);
    if (active) {
        if constexpr (MODE == FWD_RERUN) {
            // h[MP - j] = s(t0 - j)
#pragma unroll
            for (int j = 1; j <= MP; ++j) {
                S v = S(0);
                if (Xin != nullptr) v = Xin[q * MP + (j - 1)];
                else if (zi != nullptr && j <= M) v = zi[b * M + (j - 1)];
                h[MP - j] = v;
            }
        } else if constexpr (MODE == BWD_RERUN) {
            // h[j - 1] = q_j entering from the chunk's end
            if (Xin != nullptr) {
#pragma unroll
                for (int j = 0; j < MP; ++j) h[j] = Xin[q * MP + j];
            }
        }
    }
    const int nblk = L / SRS;
    S ucur[SRS], unxt[SRS];
    rec_issue_stage<S, MP, EXACT, BWD>(a_ring, bars, a, M, L, 0, active, base, n);
    rec_load_inputs<S, BWD>(ucur, u, L, 0, active, base, n);
#pragma unroll 1
    for (int s = 0; s < nblk; ++s) {
        const int slot = s & 1;
        const bool more = s + 1 < nblk;
        if (more) {
            rec_issue_stage<S, MP, EXACT, BWD>(a_ring + (slot ^ 1) * RG::A_ST, bars + (slot ^ 1), a, M, L, s + 1, active,
                                               base, n);
            rec_load_inputs<S, BWD>(unxt, u, L, s + 1, active, base, n);
        } else {
            cp_async_commit();
        }
        cp_async_wait<1>();
        if (!mbar_wait_warp(bars + slot, (s >> 1) & 1, kWaitLimit)) {
            if (lane == 0) atomicExch(status, DEV_TIMEOUT_TMA);
            if (more) mbar_wait_warp(bars + (slot ^ 1), ((s + 1) >> 1) & 1, kWaitLimit);
            cp_async_wait<0>();
            return;
        }
        __syncwarp();
        const S *ar = a_ring + slot * RG::A_ST;
        const int roff = BWD ? L - (s + 1) * SRS : s * SRS;
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
                load_pair_smem<S, MP>(c0, c1, ar + r0 * MP);
                if constexpr (MODE == FWD_RERUN) {
                    const S y0 = fwd_step_win<S, MP, WIN>(h, c0, ucur[r0], 2 * p);
                    const S y1 = fwd_step_win<S, MP, WIN>(h, c1, ucur[r0 + 1], 2 * p + 1);
                    if (roff + r0 < n) out[base + roff + r0] = y0;
                    if (roff + r0 + 1 < n) out[base + roff + r0 + 1] = y1;
                } else {
                    const S y1 = bwd_step_win<S, MP, WIN>(h, c1, ucur[r0 + 1], 2 * pr);
                    const S y0 = bwd_step_win<S, MP, WIN>(h, c0, ucur[r0], 2 * pr + 1);
                    if constexpr (MODE == BWD_RERUN) {
                        if (roff + r0 + 1 < n) out[base + roff + r0 + 1] = y1;
                        if (roff + r0 < n) out[base + roff + r0] = y0;
                    }
                }
            }
            slide<S, MP, WIN>(h);
        }
#pragma unroll
        for (int r = 0; r < SRS; ++r) ucur[r] = unxt[r];
        __syncwarp();
    }
    cp_async_wait<0>();
    if (!active) return;
    if constexpr (MODE == BWD_ZERO) {
        // adjoint zero-state summaries use the 16-byte stride of the scan's z
        constexpr int ZS = ((MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
#pragma unroll
        for (int j = 0; j < MP; ++j) Zout[q * ZS + j] = h[j];
    }
    if constexpr (MODE == BWD_RERUN) {
        if (gzi != nullptr && c == 0) {
#pragma unroll
            for (int j = 0; j < MP; ++j)
                if (j < M) gzi[b * M + j] = h[j];
        }
    }
}

// ---------------------------------------------------------------------------
// K2: cross-chunk scan in two levels.  Chunks are grouped G2 at a time by
// chunk index (group g = chunks [g*G2, (g+1)*G2)).  Along the chain the
// forward visits chunks and groups in increasing order, the adjoint in
// decreasing order.
//   k2_group   one warp per group (all signals at once):
//              CH_FWD / CH_BWD: composes the group's chunk maps x -> P x + y
//                into one map (Phi_g, y_g), stored in the chunk-map layout
//                at GY;
//              CH_TRANS: folds the adjoint's chunk maps w -> P^T w + z into
//                the group's zero-state adjoint zeta_g (GZ); the group's
//                transfer is the transpose of the forward's Phi_g.
//   k2_chain   one warp per signal: chains the groups -> the incoming state
//              of every group (GX).
//   k2_expand  one warp per group: runs the group's chunks from its incoming
//              state and writes each chunk's incoming state X (and, in the
//              forward, the checkpoints).
// Maps reach shared memory through a ring per warp filled by bulk (TMA)
// copies; when it holds a warp's whole sequence, all copies go out at once.
// Chunk map layout (stride YS): Y[0][k] = y[k], Y[r][k] = P[k][r-1].
// ---------------------------------------------------------------------------
enum { CH_FWD = 0, CH_BWD = 1, CH_TRANS = 2 };

template <typename S, int MP> struct ScanGeo {
    static constexpr int YS = YGeo<S, MP>::YS;
    static constexpr int ZS = ((MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
    static constexpr int SLOT = YS + ZS;  // a map and, for the adjoint, its z
    static_assert((YS * sizeof(S)) % 16 == 0 && (ZS * sizeof(S)) % 16 == 0, "16-byte maps");
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
// memory: straight (x -> P x + y, map at m) or transposed (w -> P^T w + z,
// P from the map at m, z at zv)
template <typename S, int MP, bool TRANS>
__device__ __forceinline__ void map_cols(S (&p)[MP + 1], const S *m, const S *zv, int j0) {
    if constexpr (TRANS) {
#pragma unroll
        for (int k = 0; k < MP; ++k) p[k + 1] = m[(j0 + 1) * MP + k];
        p[0] = zv[j0];
    } else {
#pragma unroll
        for (int r = 0; r <= MP; ++r) p[r] = m[r * MP + j0];
    }
}

// A warp's ring of `nslot` map slots filled by bulk copies.  Item i of the
// warp's sequence goes to slot i % nslot; its map comes from `map` and, for
// the adjoint, a z vector from `zvec`.  When the ring holds every item of the
// sequence, everything is issued up front and no slot is reused.
template <typename S, int MP> struct MapRing {
    using SG = ScanGeo<S, MP>;
    S *ring;
    uint64_t *bars;
    int lane, nslot;
    __device__ void init(unsigned char *base, int lane_, int nslot_) {
        nslot = nslot_;
        ring = reinterpret_cast<S *>(base);
        bars = reinterpret_cast<uint64_t *>(base + (size_t)nslot * SG::SLOT * sizeof(S));
        lane = lane_;
        if (lane == 0) {
            for (int s = 0; s < nslot; ++s) mbar_init(bars + s, 1);
            mbar_init_fence();
        }
        __syncwarp();
    }
    __device__ void issue(int i, const S *map, const S *zvec) {
        const int sl = i % nslot;
        if (lane == 0) {
            const unsigned bytes = SG::YS * sizeof(S) + (zvec ? SG::ZS * sizeof(S) : 0);
            mbar_arrive_expect_tx(bars + sl, bytes);
            bulk_load(ring + sl * SG::SLOT, map, SG::YS * sizeof(S), bars + sl);
            if (zvec) bulk_load(ring + sl * SG::SLOT + SG::YS, zvec, SG::ZS * sizeof(S), bars + sl);
        }
    }
    // nullptr when the wait gave up; the copies still in flight (items
    // i+1 .. issued-1) then get a bounded chance to land before the warp leaves
    __device__ const S *wait(int i, int issued, int *status) {
        const int sl = i % nslot;
        if (!mbar_wait_warp(bars + sl, (i / nslot) & 1, kWaitLimit)) {
            if (lane == 0) atomicExch(status, DEV_TIMEOUT_TMA);
            for (int k = i + 1; k < issued; ++k) mbar_wait_warp(bars + k % nslot, (k / nslot) & 1, kWaitLimit);
            return nullptr;
        }
        return ring + sl * SG::SLOT;
    }
};
// bytes of a warp's ring of `nslot` slots (128-byte multiple)
template <typename S, int MP> __host__ __device__ constexpr size_t ring_bytes(int nslot) {
    return ((size_t(nslot) * ScanGeo<S, MP>::SLOT * sizeof(S) + size_t(nslot) * 8 + 127) / 128) * 128;
}

constexpr int kScanWarps = 4;  // warps per block of k2_group / k2_expand

template <typename S, int MP, int MODE>
__global__ void __launch_bounds__(kScanWarps * 32)
    k2_group(int64_t nC, int G2, int nG, int64_t n_items, int nslot, const S *__restrict__ Y,
             const S *__restrict__ Z, S *__restrict__ GY, S *__restrict__ GZ, int *__restrict__ status) {
    using SG = ScanGeo<S, MP>;
    constexpr int YS = SG::YS, ZS = SG::ZS;
    constexpr bool REV = MODE != CH_FWD;
    constexpr bool TRANS = MODE == CH_TRANS;
    extern __shared__ __align__(128) unsigned char k2g_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kScanWarps + warp;  // b * nG + g
    if (item >= n_items) return;
    const int64_t b = item / nG;
    const int g = (int)(item - b * nG);
    MapRing<S, MP> R;
    R.init(k2g_smem + (size_t)warp * ring_bytes<S, MP>(nslot), lane, nslot);
    const int64_t c_lo = (int64_t)g * G2;
    const int len = (int)((c_lo + G2 <= nC ? c_lo + G2 : nC) - c_lo);
    auto chunk_at = [&](int i) -> int64_t { return b * nC + (REV ? c_lo + len - 1 - i : c_lo + i); };
    int issued = 0;
    auto issue = [&](int i) {
        if (i < len) {
            R.issue(i, Y + chunk_at(i) * YS, TRANS ? Z + chunk_at(i) * ZS : nullptr);
            issued = i + 1;
        }
    };
    for (int i = 0; i < nslot - 1 || (nslot >= len && i < len); ++i) issue(i);
    const int j0 = lane < MP ? lane : 0;
    if constexpr (TRANS) {
        S zeta = S(0);
        for (int i = 0; i < len; ++i) {
            const S *m = R.wait(i, issued, status);
            if (m == nullptr) return;
            S p[MP + 1];
            map_cols<S, MP, true>(p, m, m + YS, j0);
            __syncwarp();
            if (nslot < len) issue(i + nslot - 1);
            zeta = hop<S, MP>(p, zeta, lane);
        }
        if (lane < MP) GZ[item * ZS + lane] = zeta;
    } else {
        // lane j < MP holds column j of the composed transfer (its response
        // to a unit incoming component j+1); the accumulated response y is
        // folded by a hop chain, one component per lane
        S col[MP];
#pragma unroll
        for (int k = 0; k < MP; ++k) col[k] = (k == lane) ? S(1) : S(0);
        S yv = S(0);
        for (int i = 0; i < len; ++i) {
            const S *m = R.wait(i, issued, status);
            if (m == nullptr) return;
            S p[MP + 1];
            map_cols<S, MP, false>(p, m, nullptr, j0);
            S acc[MP];
#pragma unroll
            for (int k = 0; k < MP; ++k) acc[k] = S(0);
#pragma unroll
            for (int r = 1; r <= MP; ++r) {
                const S xr = col[r - 1];
                const S *row = m + r * MP;  // P[k][r-1] = m[r*MP + k]
#pragma unroll
                for (int k = 0; k < MP; k += 2) {
                    if constexpr (sizeof(S) == 4) {
                        const float2 v = *reinterpret_cast<const float2 *>(row + k);
                        acc[k] = fma((S)v.x, xr, acc[k]);
                        acc[k + 1] = fma((S)v.y, xr, acc[k + 1]);
                    } else {
                        acc[k] = fma(row[k], xr, acc[k]);
                        acc[k + 1] = fma(row[k + 1], xr, acc[k + 1]);
                    }
                }
            }
            __syncwarp();
            if (nslot < len) issue(i + nslot - 1);
            yv = hop<S, MP>(p, yv, lane);
#pragma unroll
            for (int k = 0; k < MP; ++k) col[k] = acc[k];
        }
        if (lane < MP) {
            GY[item * YS + lane] = yv;
#pragma unroll
            for (int k = 0; k < MP; ++k) GY[item * YS + (lane + 1) * MP + k] = col[k];
        }
    }
}

template <typename S, int MP, int MODE>
__global__ void __launch_bounds__(32)
    k2_chain(int M, int nG, int nslot, const S *__restrict__ GY, const S *__restrict__ GZ, const S *__restrict__ zi,
             S *__restrict__ GX, int *__restrict__ status) {
    using SG = ScanGeo<S, MP>;
    constexpr int YS = SG::YS, ZS = SG::ZS;
    constexpr bool REV = MODE != CH_FWD;
    constexpr bool TRANS = MODE == CH_TRANS;
    extern __shared__ __align__(128) unsigned char k2c_smem[];
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x;
    MapRing<S, MP> R;
    R.init(k2c_smem, lane, nslot);
    auto gof = [&](int n) -> int64_t { return b * nG + (REV ? nG - 1 - n : n); };
    int issued = 0;
    auto issue = [&](int n) {
        // the last group's map is not needed: nothing follows it
        if (n < nG - 1) {
            R.issue(n, GY + gof(n) * YS, TRANS ? GZ + gof(n) * ZS : nullptr);
            issued = n + 1;
        }
    };
    for (int n = 0; n < nslot - 1 || (nslot >= nG - 1 && n < nG - 1); ++n) issue(n);
    const int j0 = lane < MP ? lane : 0;
    S x = S(0);
    if (MODE == CH_FWD && zi != nullptr && lane < M) x = zi[b * M + lane];
    for (int n = 0; n < nG; ++n) {
        if (lane < MP) GX[gof(n) * ZS + lane] = x;
        if (n == nG - 1) break;
        const S *m = R.wait(n, issued, status);
        if (m == nullptr) return;
        S p[MP + 1];
        map_cols<S, MP, TRANS>(p, m, m + YS, j0);
        __syncwarp();
        if (nslot < nG - 1) issue(n + nslot - 1);
        x = hop<S, MP>(p, x, lane);
    }
}

template <typename S, int MP, int MODE>
__global__ void __launch_bounds__(kScanWarps * 32)
    k2_expand(int M, int64_t nC, int G2, int nG, int64_t n_items, int nslot, const S *__restrict__ Y,
              const S *__restrict__ Z, const S *__restrict__ GX, S *__restrict__ X, S *__restrict__ ckpt,
              int *__restrict__ status) {
    using SG = ScanGeo<S, MP>;
    constexpr int YS = SG::YS, ZS = SG::ZS;
    constexpr bool REV = MODE != CH_FWD;
    constexpr bool TRANS = MODE == CH_TRANS;
    extern __shared__ __align__(128) unsigned char k2e_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kScanWarps + warp;  // b * nG + g
    if (item >= n_items) return;
    const int64_t b = item / nG;
    const int g = (int)(item - b * nG);
    MapRing<S, MP> R;
    R.init(k2e_smem + (size_t)warp * ring_bytes<S, MP>(nslot), lane, nslot);
    const int64_t c_lo = (int64_t)g * G2;
    const int len = (int)((c_lo + G2 <= nC ? c_lo + G2 : nC) - c_lo);
    auto chunk_at = [&](int i) -> int64_t { return REV ? c_lo + len - 1 - i : c_lo + i; };
    int issued = 0;
    auto issue = [&](int i) {
        // the group's last chunk needs no map: nothing follows it in the group
        if (i < len - 1) {
            R.issue(i, Y + (b * nC + chunk_at(i)) * YS, TRANS ? Z + (b * nC + chunk_at(i)) * ZS : nullptr);
            issued = i + 1;
        }
    };
    for (int i = 0; i < nslot - 1 || (nslot >= len - 1 && i < len - 1); ++i) issue(i);
    const int j0 = lane < MP ? lane : 0;
    S x = lane < MP ? GX[item * ZS + lane] : S(0);
    for (int i = 0; i < len; ++i) {
        const int64_t c = chunk_at(i);
        if (lane < MP) X[(b * nC + c) * MP + lane] = x;
        if (MODE == CH_FWD && ckpt != nullptr && lane < M) ckpt[(b * nC + c) * M + lane] = x;
        if (i == len - 1) break;
        const S *m = R.wait(i, issued, status);
        if (m == nullptr) return;
        S p[MP + 1];
        map_cols<S, MP, TRANS>(p, m, m + YS, j0);
        __syncwarp();
        if (nslot < len - 1) issue(i + nslot - 1);
        x = hop<S, MP>(p, x, lane);
    }
}

// ---------------------------------------------------------------------------
// Coefficient gradient (Eq. 12): ga[b][t][i-1] = -ge(b,t) * s(b, t-i), with
// s(b, -j) = zi[b][j-1] (zero without zi).  A block owns TR rows of one
// signal: it stages ge and the s window in shared memory, then writes its
// TR*M outputs, one contiguous span, with 16-byte stores when aligned.
// ---------------------------------------------------------------------------
template <typename S, int MP, bool EXACT> struct GradGeo {
    static constexpr int TR = 256;       // rows per block
    static constexpr int THREADS = 256;
};

template <typename S, int MP, bool EXACT>
__global__ void __launch_bounds__(256)
    k_grad_a(int64_t T, int M, int64_t tiles_per_signal, const S *__restrict__ ge, const S *__restrict__ s,
             const S *__restrict__ zi, S *__restrict__ ga) {
    constexpr int TR = GradGeo<S, MP, EXACT>::TR;
    __shared__ S g_t[TR];
    __shared__ S s_t[TR + MP];
    const int64_t b = blockIdx.x / tiles_per_signal;
    const int64_t t0 = (blockIdx.x - b * tiles_per_signal) * (int64_t)TR;
    const int rows = (T - t0) < TR ? (int)(T - t0) : TR;
    const int Mc = EXACT ? MP : M;
    for (int i = threadIdx.x; i < TR + MP; i += blockDim.x) {
        const int64_t t = t0 - MP + i;  // s_t[i] = s(t0 - MP + i)
        S v = S(0);
        if (t >= 0 && t < T) v = s[b * T + t];
        else if (t < 0 && zi != nullptr && -t <= M) v = zi[b * M + (-t - 1)];
        s_t[i] = v;
        if (i < TR) g_t[i] = (i < rows) ? ge[b * T + t0 + i] : S(0);
    }
    __syncthreads();
    S *dst = ga + (b * T + t0) * (int64_t)Mc;
    const int total = rows * Mc;
    const bool vec = sizeof(S) == 4 && aligned16(dst);
    if (vec) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        const int n4 = total / 4;
        for (int v = threadIdx.x; v < n4; v += blockDim.x) {
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int idx = 4 * v + e;
                const int r = idx / Mc, i = idx - r * Mc;  // i = coefficient index - 1
                o[e] = (float)(-g_t[r] * s_t[MP + r - (i + 1)]);
            }
            d4[v] = make_float4(o[0], o[1], o[2], o[3]);
        }
        for (int idx = 4 * n4 + threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = idx / Mc, i = idx - r * Mc;
            dst[idx] = -g_t[r] * s_t[MP + r - (i + 1)];
        }
    } else {
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = idx / Mc, i = idx - r * Mc;
            dst[idx] = -g_t[r] * s_t[MP + r - (i + 1)];
        }
    }
}

}  // namespace tvlp
