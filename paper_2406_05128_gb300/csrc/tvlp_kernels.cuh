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
// Parallel scan over time.  A signal is cut into chunks of L samples.
//   k1_summary      per chunk, the end states of MP+1 recursions: zero state
//                   driven by the input (column 0) and the MP unit initial
//                   states with zero input (columns 1..MP, the chunk transfer
//                   P_c).  Forward direction; also available backwards.
//   k_rec (ZERO)    per chunk, one recursion from zero state; end state only
//                   (the adjoint's zero-state summary z_c).
//   k2_chain        x_{c+1} = P_c x_c + y_c (forward) or
//                   w_{c-1} = P_c^T w_c + z_c (adjoint) per signal.
//   k_rec (RERUN)   each chunk re-runs its recursion from its true incoming
//                   state and writes s (forward) or ge (adjoint).  With one
//                   chunk per signal this is the plain sequential filter.
//   k_grad_a        dL/da_i(t) = -ge(t) s(t-i) (Eq. 12), tiled.
// Orders are padded to MP (compile time); coefficients of order > M are
// zero, which leaves every result unchanged.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tvlp {

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

template <typename S, int MP> struct Geo {
    static constexpr int G = Pack<MP>::G;
    static constexpr int R = Pack<MP>::R;
    static constexpr int CPW = 32 / G;                     // chunks per warp
    static constexpr int NS = 2;                            // stages in flight
    static constexpr int WPS = (int)sizeof(S) / 4;          // 32-bit words per element
    static constexpr int GPH = (16 / G) > 1 ? 16 / G : 1;   // chunk groups per half-warp
    // chunk-stage stride (elements): MP rows of MP coefficients + padding,
    // a multiple of 16 bytes (TMA destination alignment)
    static constexpr int CS = MP * MP + conflict_free_pad(MP * MP * WPS, GPH, 4) / WPS;
    static constexpr int US = MP + 1;                        // input stride per chunk-stage
    static constexpr int A_STAGE = CPW * CS;
    static constexpr int U_STAGE = ((CPW * US + 3) / 4) * 4;
    static constexpr int WARP_ELEMS = NS * (A_STAGE + U_STAGE);
    static constexpr size_t WARP_BYTES = size_t(WARP_ELEMS) * sizeof(S) + NS * 8;  // + mbarriers
    // per-chunk stride of the summaries Y[c][MP+1][MP], a multiple of 16 bytes
    static constexpr int YS = (((MP + 1) * MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
    static_assert(G * R >= MP + 1, "packing must hold MP+1 recursions");
    static_assert((CS * sizeof(S)) % 16 == 0, "chunk stage must stay 16-byte aligned");
    static_assert((WARP_ELEMS * sizeof(S)) % 16 == 0, "warp region must stay 16-byte aligned");
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
// Bounded wait for an mbarrier phase; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__host__ __device__ constexpr int wrapm(int x, int m) { return ((x % m) + m) % m; }

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

// Forward direct-form step at chunk-local time t with t % MP == TT:
// h[t % MP] holds s(t).  Four partial sums over the older terms, then the
// two freshest outputs, keep the critical path to a few FMAs per step.
template <typename S, int MP>
__device__ __forceinline__ S fwd_step(S (&h)[MP], const S (&c)[MP], S u, int tt) {
    S p0 = u, p1 = S(0), p2 = S(0), p3 = S(0);
#pragma unroll
    for (int i = MP; i >= 3; --i) {
        const S hv = h[wrapm(tt - i, MP)];
        if ((i & 3) == 0) p0 = fma(-c[i - 1], hv, p0);
        else if ((i & 3) == 1) p1 = fma(-c[i - 1], hv, p1);
        else if ((i & 3) == 2) p2 = fma(-c[i - 1], hv, p2);
        else p3 = fma(-c[i - 1], hv, p3);
    }
    S acc = (p0 + p1) + (p2 + p3);
    if constexpr (MP >= 2) acc = fma(-c[1], h[wrapm(tt - 2, MP)], acc);
    acc = fma(-c[0], h[wrapm(tt - 1, MP)], acc);
    h[tt] = acc;
    return acc;
}

// Backward transposed-form step: q_1 sits in slot p and q_k in slot
// (p + k - 1) % MP before the step; after it q_k sits in (p + k) % MP.
template <typename S, int MP>
__device__ __forceinline__ S bwd_step(S (&q)[MP], const S (&c)[MP], S u, int p) {
    const S y = u + q[p];
    q[p] = -c[MP - 1] * y;
#pragma unroll
    for (int k = 1; k < MP; ++k) q[wrapm(p + k, MP)] = fma(-c[k - 1], y, q[wrapm(p + k, MP)]);
    return y;
}

// ---------------------------------------------------------------------------
// K1: chunk summaries.
// Flattened chunk index q = b*nC + c; chunk c of signal b covers samples
// [c*L, c*L + L); rows at or beyond T read as zero (exact: the forward's
// last chunk has no successor; in the adjoint, zero input and coefficients
// past T keep the pending state at zero).
// Each warp owns CPW consecutive chunks; lane (grp = lane/G, g = lane%G)
// runs recursions r = g*R + k, k < R.  Coefficient rows are staged through
// shared memory, MP rows per stage, two stages in flight: full chunk-stages
// arrive by one 1-D bulk (TMA) copy each, completing on a per-stage
// mbarrier; ragged or misaligned chunk-stages and the input samples use
// cp.async with zero fill.  Forward stages advance in time, backward stages
// go back in time.
// Output Y[q][r][k] (per-chunk stride YS):
//   forward:  s(c*L + L - 1 - k) of recursion r
//   backward: q_{k+1} after the chunk, i.e. the pending dL/ds(c*L - 1 - k)
// ---------------------------------------------------------------------------
template <typename S, int MP, bool BWD>
__device__ __forceinline__ void k1_issue_stage(S *a_st, S *u_st, uint64_t *bar, const S *__restrict__ a,
                                               const S *__restrict__ u, int M, int L, int k, int lane,
                                               int64_t my_base, int my_valid, bool exact) {
    using GE = Geo<S, MP>;
    constexpr int CPW = GE::CPW;
    constexpr unsigned STAGE_BYTES = MP * MP * sizeof(S);
    const int roff = BWD ? L - (k + 1) * MP : k * MP;  // chunk-local first row of the stage
    // lane ch < CPW describes chunk ch
    int nvalid = my_valid - roff;
    nvalid = nvalid < 0 ? 0 : (nvalid > MP ? MP : nvalid);
    const S *src = a + (my_base + roff) * (int64_t)MP;
    bool tma = false;
    if (lane < CPW) tma = exact && nvalid == MP && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
    const unsigned tma_mask = __ballot_sync(0xffffffffu, tma);
    if (lane == 0) mbar_arrive_expect_tx(bar, __popc(tma_mask) * STAGE_BYTES);
    __syncwarp();
    if (tma) {
        fence_proxy_async();
        bulk_load(a_st + lane * GE::CS, src, STAGE_BYTES, bar);
    }
    // fallback chunk-stages (ragged tail, misaligned start, padded order)
    unsigned slow = __ballot_sync(0xffffffffu, lane < CPW && !tma) & ((1u << CPW) - 1u);
    while (slow) {
        const int ch = __ffs(slow) - 1;
        slow &= slow - 1;
        const int64_t base = __shfl_sync(0xffffffffu, my_base, ch);
        const int nv = __shfl_sync(0xffffffffu, nvalid, ch);
        S *dst = a_st + ch * GE::CS;
        if (exact) {
            const S *s0 = a + (base + roff) * (int64_t)MP;
            for (int idx = lane; idx < MP * MP; idx += 32) {
                const bool v = idx < nv * MP;
                cp_async<sizeof(S)>(dst + idx, v ? s0 + idx : a, v ? (int)sizeof(S) : 0);
            }
        } else {
            for (int r = 0; r < MP; ++r) {
                if (lane < M) {
                    const bool v = r < nv;
                    const S *s0 = v ? a + (base + roff + r) * (int64_t)M + lane : a;
                    cp_async<sizeof(S)>(dst + r * MP + lane, s0, v ? (int)sizeof(S) : 0);
                }
            }
        }
    }
    // input samples of every chunk-stage (lane r copies row r)
#pragma unroll 1
    for (int ch = 0; ch < CPW; ++ch) {
        const int64_t base = __shfl_sync(0xffffffffu, my_base, ch);
        const int nv = __shfl_sync(0xffffffffu, nvalid, ch);
        if (lane < MP) {
            const bool v = lane < nv;
            cp_async<sizeof(S)>(u_st + ch * GE::US + lane, v ? u + base + roff + lane : u, v ? (int)sizeof(S) : 0);
        }
    }
    cp_async_commit();
}

template <typename S, int MP, bool BWD>
__global__ void __launch_bounds__(256, 1)
    k1_summary(int64_t T, int M, int L, int64_t nC, int64_t NQ, const S *__restrict__ a, const S *__restrict__ u,
               S *__restrict__ Y, int exact_flag, int *__restrict__ status) {
    using GE = Geo<S, MP>;
    constexpr int G = GE::G, R = GE::R, CPW = GE::CPW;
    extern __shared__ __align__(128) unsigned char k1_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t q0 = ((int64_t)blockIdx.x * wpb + warp) * CPW;
    if (q0 >= NQ) return;
    const bool exact = exact_flag != 0;
    unsigned char *wbase = k1_smem + (size_t)warp * GE::WARP_BYTES;
    S *a_buf = reinterpret_cast<S *>(wbase);                 // [NS][A_STAGE]
    S *u_buf = a_buf + GE::NS * GE::A_STAGE;                  // [NS][U_STAGE]
    uint64_t *bars = reinterpret_cast<uint64_t *>(u_buf + GE::NS * GE::U_STAGE);
    if (!exact) {
        for (int idx = lane; idx < GE::NS * GE::A_STAGE; idx += 32) a_buf[idx] = S(0);
    }
    if (lane == 0) {
        for (int s = 0; s < GE::NS; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    // lane ch < CPW describes chunk q0 + ch: first row b*T + c*L and valid rows
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
    const int nblk = L / MP;

    // forward: h[k][t % MP] = output of recursion k at chunk-local time t
    // backward: h[k][slot] = pending state (q_j in slot j % MP at start)
    S h[R][MP];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = g * R + k;
#pragma unroll
        for (int m = 0; m < MP; ++m) {
            const int unit_slot = BWD ? (r % MP) : ((MP - (r % MP)) % MP);
            h[k][m] = (r >= 1 && r <= MP && m == unit_slot) ? S(1) : S(0);
        }
    }
    const S flag0 = (g == 0) ? S(1) : S(0);

    k1_issue_stage<S, MP, BWD>(a_buf, u_buf, bars, a, u, M, L, 0, lane, my_base, my_valid, exact);
#pragma unroll 1
    for (int k = 0; k < nblk; ++k) {
        const int slot = k & 1;
        if (k + 1 < nblk)
            k1_issue_stage<S, MP, BWD>(a_buf + (slot ^ 1) * GE::A_STAGE, u_buf + (slot ^ 1) * GE::U_STAGE,
                                       bars + (slot ^ 1), a, u, M, L, k + 1, lane, my_base, my_valid, exact);
        else
            cp_async_commit();
        cp_async_wait<1>();
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(bars + slot, (k >> 1) & 1, 1 << 22) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            // a bulk copy never completed: record it, give the copy in flight
            // for the other stage a bounded chance to land, and leave
            if (lane == 0) {
                atomicExch(status, DEV_TIMEOUT_TMA);
                if (k + 1 < nblk) mbar_wait_bounded(bars + (slot ^ 1), ((k + 1) >> 1) & 1, 1 << 22);
            }
            cp_async_wait<0>();
            __syncwarp();
            return;
        }
        __syncwarp();
        const S *arow = a_buf + slot * GE::A_STAGE + grp * GE::CS;
        const S *urow = u_buf + slot * GE::U_STAGE + grp * GE::US;
#pragma unroll
        for (int step = 0; step < MP; ++step) {
            // forward: row tt = step (t % MP == tt); backward: row tt = MP-1-step,
            // and q_1 sits in slot (step + 1) % MP
            const int tt = BWD ? MP - 1 - step : step;
            S c[MP];
            load_row_smem<S, MP>(c, arow + tt * MP);
            const S uu = flag0 * urow[tt];
            if constexpr (BWD) {
                const int p = (step + 1) % MP;
                S y[R];
#pragma unroll
                for (int kk = 0; kk < R; ++kk) y[kk] = ((kk == 0) ? uu : S(0)) + h[kk][p];
#pragma unroll
                for (int kk = 0; kk < R; ++kk) h[kk][p] = -c[MP - 1] * y[kk];
#pragma unroll
                for (int j = 1; j < MP; ++j)
#pragma unroll
                    for (int kk = 0; kk < R; ++kk) h[kk][(p + j) % MP] = fma(-c[j - 1], y[kk], h[kk][(p + j) % MP]);
            } else {
                S acc[R];
#pragma unroll
                for (int kk = 0; kk < R; ++kk) acc[kk] = (kk == 0) ? uu : S(0);
#pragma unroll
                for (int i = MP; i >= 1; --i)
#pragma unroll
                    for (int kk = 0; kk < R; ++kk) acc[kk] = fma(-c[i - 1], h[kk][wrapm(tt - i, MP)], acc[kk]);
#pragma unroll
                for (int kk = 0; kk < R; ++kk) h[kk][tt] = acc[kk];
            }
        }
        __syncwarp();
    }
    // end states
    const int64_t q = q0 + grp;
    if (q < NQ) {
        S *yq = Y + q * GE::YS;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int r = g * R + k;
            if (r <= MP) {
#pragma unroll
                for (int j = 0; j < MP; ++j) {
                    // forward: s(L-1-j) sits in slot (MP-1-j); backward: q_{j+1} in (j+1) % MP
                    const int sl = BWD ? (j + 1) % MP : MP - 1 - j;
                    yq[r * MP + j] = h[k][sl];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// One recursion per thread over its chunk ("lane per chunk").  Coefficient
// rows and input samples stream through a private shared-memory ring of D
// rows per thread, filled by cp.async D-2 rows ahead, two rows per group.
//   FWD_RERUN: start from X[q] (or zi / zero), write s.
//   BWD_ZERO:  adjoint from zero state, store the end state to Z[q].
//   BWD_RERUN: adjoint from W[q], write ge; chunk 0 also writes gzi.
// A launch with one chunk per signal (L >= T) is the plain sequential filter.
// Blocks walk the chunks in reverse order when `reverse` is set, so that a
// pass right after another one over the same rows starts with the rows that
// pass loaded last (most likely still in L2).
// ---------------------------------------------------------------------------
enum { FWD_RERUN = 0, BWD_ZERO = 1, BWD_RERUN = 2 };

template <typename S, int MP> struct RingGeo {
    static constexpr int D = 16;                       // rows per thread ring (power of two)
    static constexpr int SLOT = MP + 2;                // MP coefficients, input, pad (elements)
    static constexpr int WPS = (int)sizeof(S) / 4;
    static constexpr int RAW = D * SLOT * WPS;         // words per thread
    // thread stride in words, 2*WPS mod 32, so 8-byte (float) / 16-byte
    // (double) row loads of a half / quarter warp hit distinct banks
    static constexpr int TW = RAW + wrapm(2 * WPS - RAW, 32);
    static constexpr int THREADS = 32;
    static constexpr size_t SMEM = size_t(THREADS) * TW * 4;
};

template <typename S, int MP, bool EXACT>
__device__ __forceinline__ void ring_issue_row(S *slot, const S *__restrict__ row, const S *__restrict__ up,
                                               int M) {
    if constexpr (EXACT) {
        // M == MP: the row is MP contiguous elements, 8-byte aligned
#pragma unroll
        for (int j = 0; j < MP * (int)sizeof(S) / 8; ++j)
            cp_async<8>(reinterpret_cast<char *>(slot) + 8 * j, reinterpret_cast<const char *>(row) + 8 * j, 8);
    } else {
        for (int j = 0; j < M; ++j) cp_async<sizeof(S)>(slot + j, row + j, (int)sizeof(S));
    }
    cp_async<sizeof(S)>(slot + MP, up, (int)sizeof(S));
}

template <typename S, int MP, bool EXACT, int MODE>
__global__ void __launch_bounds__(32)
    k_rec(int64_t T, int M, int L, int64_t nC, int64_t NQ, const S *__restrict__ a, const S *__restrict__ u,
          const S *__restrict__ Xin, const S *__restrict__ zi, S *__restrict__ out, S *__restrict__ Zout,
          S *__restrict__ gzi, int reverse) {
    using RG = RingGeo<S, MP>;
    constexpr int D = RG::D, SLOT = RG::SLOT;
    constexpr bool BWD = MODE != FWD_RERUN;
    extern __shared__ __align__(16) unsigned char rec_smem[];
    const int64_t blk = reverse ? (int64_t)gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int64_t q = blk * RG::THREADS + threadIdx.x;
    if (q >= NQ) return;
    S *ring = reinterpret_cast<S *>(rec_smem + (size_t)threadIdx.x * RG::TW * 4);
    if (!EXACT) {
        for (int j = 0; j < D * SLOT; ++j) ring[j] = S(0);
    }
    const int64_t b = q / nC;
    const int64_t c = q - b * nC;
    const int64_t t0 = c * (int64_t)L;
    const int64_t rem = T - t0;
    const int n = rem < L ? (int)rem : L;  // valid rows of this chunk
    const S *arow = a + (b * T + t0) * (int64_t)M;
    const S *up = u + b * T + t0;

    S h[MP];
    if constexpr (MODE == FWD_RERUN) {
        // s(t0-1-j) sits in slot (t0-1-j) % MP = MP-1-j  (t0 is a multiple of MP)
#pragma unroll
        for (int j = 0; j < MP; ++j) {
            S v = S(0);
            if (Xin != nullptr) v = Xin[q * MP + j];
            else if (zi != nullptr && j < M) v = zi[b * M + j];
            h[MP - 1 - j] = v;
        }
    } else {
        // pending state entering from the chunk's end: q_j in slot j % MP
#pragma unroll
        for (int j = 1; j <= MP; ++j) h[j % MP] = (MODE == BWD_RERUN && Xin != nullptr) ? Xin[q * MP + (j - 1)] : S(0);
    }

    // valid rows in processing order: forward t0, t0+1, ...; backward
    // t0+n-1, ..., t0.  Row r of that order sits in ring slot r % D.
    auto row_of = [&](int r) -> int { return BWD ? n - 1 - r : r; };
    int nx = 0;  // next row to issue
    auto issue_upto = [&](int last) {
        const int hi = last < n - 1 ? last : n - 1;
        for (; nx <= hi; ++nx) {
            const int lr = row_of(nx);
            ring_issue_row<S, MP, EXACT>(ring + (nx & (D - 1)) * SLOT, arow + (int64_t)lr * M, up + lr, M);
        }
        cp_async_commit();
    };
    // prologue: rows 0..D-3, two per group
#pragma unroll 1
    for (int g = 0; g < (D - 2) / 2; ++g) issue_upto(2 * g + 1);
    // Nominal steps run over the whole chunk (L, a multiple of MP) so the
    // rotation phases are compile-time constants; rows beyond T are skipped
    // (only in the last chunk, where they sit after the forward's last valid
    // row or before the adjoint's first one, with a zero pending state).
    const int skip = BWD ? L - n : 0;  // nominal steps before the first valid row
    int r = 0;                          // valid rows processed so far
    auto one_step = [&](const S(&cc)[MP], S uu, int step) {
        const int lr = row_of(r);
        if constexpr (MODE == FWD_RERUN) {
            out[b * T + t0 + lr] = fwd_step<S, MP>(h, cc, uu, step);
        } else {
            const S y = bwd_step<S, MP>(h, cc, uu, (step + 1) % MP);
            if constexpr (MODE == BWD_RERUN) out[b * T + t0 + lr] = y;
        }
        ++r;
    };
    const int nblk = L / MP;
#pragma unroll 1
    for (int bk = 0; bk < nblk; ++bk) {
        if (!BWD && bk * MP >= n) break;
        if (BWD && (bk + 1) * MP <= skip) continue;
#pragma unroll
        for (int st = 0; st < MP; st += 2) {
            const int nom0 = bk * MP + st;  // nominal step index of the pair's first step
            const bool v0 = BWD ? (nom0 >= skip) : (nom0 < n);
            const bool v1 = BWD ? (nom0 + 1 >= skip) : (nom0 + 1 < n);
            if (!v0 && !v1) continue;
            // refill up to D-1 rows ahead (slots of rows already consumed),
            // one cp.async group per pair; then wait for this pair's rows
            issue_upto(r + D - 1);
            cp_async_wait<(D - 2) / 2>();
            const S *s0 = ring + (r & (D - 1)) * SLOT;
            if (v0 && v1) {
                const S *s1 = ring + ((r + 1) & (D - 1)) * SLOT;
                S c0[MP], c1[MP];
                load_row_smem<S, MP>(c0, s0);
                load_row_smem<S, MP>(c1, s1);
                const S u0 = s0[MP], u1 = s1[MP];
                one_step(c0, u0, st);
                one_step(c1, u1, st + 1);
            } else {
                // a lone row: the forward's last row or the adjoint's first
                S c0[MP];
                load_row_smem<S, MP>(c0, s0);
                if (v0) one_step(c0, s0[MP], st);
                else one_step(c0, s0[MP], st + 1);
            }
        }
    }
    cp_async_wait<0>();
    if constexpr (MODE == BWD_ZERO) {
        // after L nominal steps (a multiple of MP) q_j is back in slot j % MP
#pragma unroll
        for (int j = 1; j <= MP; ++j) Zout[q * MP + (j - 1)] = h[j % MP];
    }
    if constexpr (MODE == BWD_RERUN) {
        if (gzi != nullptr && c == 0) {
#pragma unroll
            for (int j = 1; j <= MP; ++j)
                if (j <= M) gzi[b * M + (j - 1)] = h[j % MP];
        }
    }
}

// ---------------------------------------------------------------------------
// K2: cross-chunk chain, one warp per signal.  Lane j (< MP) holds state
// component j+1.  Summaries of upcoming chunks are prefetched into shared
// memory NB chunks ahead and into registers one chunk ahead.
//   CH_FWD:   X[b][0] = zi (0 if none); X[b][c+1] = Y0[c] + P[c] X[b][c]
//   CH_BWD:   W[b][nC-1] = 0;  W[b][c-1] = Y0[c] + P[c] W[b][c]   (adjoint's
//             own summaries, P in the pending-state basis)
//   CH_TRANS: W[b][nC-1] = 0;  W[b][c-1] = Z[c] + P[c]^T W[b][c]  (forward
//             transfers, transposed; Z the adjoint's zero-state summaries)
// X/W hold the incoming state of each chunk (stride MP).  The forward also
// writes the chunk checkpoints ckpt[b][c][0..M-1] when asked.
// ---------------------------------------------------------------------------
enum { CH_FWD = 0, CH_BWD = 1, CH_TRANS = 2 };

template <typename S, int MP> struct ChainGeo {
    static constexpr int NB = 8;                                       // chunks prefetched
    static constexpr int ZS = ((MP * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
    static constexpr int SLOT = Geo<S, MP>::YS + ZS;                   // Y block + z vector
    static constexpr size_t SMEM = size_t(NB) * SLOT * sizeof(S);
};

template <typename S, int MP, int MODE>
__global__ void __launch_bounds__(32)
    k2_chain(int B, int M, int64_t nC, const S *__restrict__ Y, const S *__restrict__ Z, const S *__restrict__ zi,
             S *__restrict__ X, S *__restrict__ ckpt) {
    using GE = Geo<S, MP>;
    using CG = ChainGeo<S, MP>;
    constexpr int NB = CG::NB;
    constexpr int YS = GE::YS;
    constexpr bool REV = MODE != CH_FWD;
    extern __shared__ __align__(16) unsigned char k2_smem[];
    S *ybuf = reinterpret_cast<S *>(k2_smem);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    if (b >= B) return;
    const S *Yb = Y + (int64_t)b * nC * YS;
    const int j0 = lane < MP ? lane : 0;

    auto chunk_of = [&](int64_t n) -> int64_t { return REV ? nC - 1 - n : n; };
    // one cp.async group per chunk: its Y block (16-byte pieces) and, for
    // the transposed chain, the adjoint's zero-state vector z
    auto issue = [&](int64_t n) {
        if (n < nC) {
            const int64_t c = chunk_of(n);
            const S *src = Yb + c * YS;
            S *dst = ybuf + (n % NB) * CG::SLOT;
            constexpr int nbytes = YS * (int)sizeof(S);
            for (int off = lane * 16; off < nbytes; off += 32 * 16)
                cp_async<16>(reinterpret_cast<char *>(dst) + off, reinterpret_cast<const char *>(src) + off, 16);
            if (MODE == CH_TRANS && lane < MP)
                cp_async<sizeof(S)>(dst + YS + lane, Z + ((int64_t)b * nC + c) * MP + lane, (int)sizeof(S));
        }
        cp_async_commit();
    };
    // the lane's coefficients for chunk n: p[0] constant term, p[r] factor of x[r-1]
    auto load_cols = [&](int64_t n, S (&p)[MP + 1]) {
        const S *yc = ybuf + (n % NB) * CG::SLOT;
        if constexpr (MODE == CH_TRANS) {
            // w_new[j] = z[j] + sum_k P[k][j] w[k],  P[k][j] = Y[j+1][k]
#pragma unroll
            for (int k = 0; k < MP; ++k) p[k + 1] = yc[(j0 + 1) * MP + k];
            p[0] = yc[YS + j0];
        } else {
            // x_new[j] = Y[0][j] + sum_r Y[r][j] x[r-1]
#pragma unroll
            for (int r = 0; r <= MP; ++r) p[r] = yc[r * MP + j0];
        }
    };

    for (int n = 0; n < NB - 1; ++n) issue(n);
    S x = S(0);
    if (MODE == CH_FWD && zi != nullptr && lane < M) x = zi[(int64_t)b * M + lane];
    S p[MP + 1];
    cp_async_wait<NB - 2>();  // chunk 0 landed
    __syncwarp();
    load_cols(0, p);
#pragma unroll 1
    for (int64_t n = 0; n < nC; ++n) {
        const int64_t c = chunk_of(n);
        if (lane < MP) X[((int64_t)b * nC + c) * MP + lane] = x;
        if (MODE == CH_FWD && ckpt != nullptr && lane < M) ckpt[((int64_t)b * nC + c) * M + lane] = x;
        if (n == nC - 1) break;
        S a0 = p[0], a1 = S(0), a2 = S(0), a3 = S(0);
#pragma unroll
        for (int r = 1; r <= MP; ++r) {
            const S xr = __shfl_sync(0xffffffffu, x, r - 1);
            if ((r & 3) == 0) a0 = fma(p[r], xr, a0);
            else if ((r & 3) == 1) a1 = fma(p[r], xr, a1);
            else if ((r & 3) == 2) a2 = fma(p[r], xr, a2);
            else a3 = fma(p[r], xr, a3);
        }
        // chunk n+1 landed once NB-2 groups at most are pending; its slot
        // refill (chunk n+NB-1) reuses the slot of chunk n-1, read already
        issue(n + NB - 1);
        cp_async_wait<NB - 2>();
        __syncwarp();
        load_cols(n + 1, p);
        x = lane < MP ? (a0 + a1) + (a2 + a3) : S(0);
    }
    cp_async_wait<0>();
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
    const bool vec = sizeof(S) == 4 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
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
