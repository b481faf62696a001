/*
 * tvlp.h — C ABI of the GB300 (sm_103a) time-varying linear-prediction
 * library.
 *
 * The library computes the sample-wise time-varying all-pole (LP) filter of
 * Yu & Fazekas, "Differentiable Time-Varying Linear Prediction in the
 * Context of End-to-End Analysis-by-Synthesis" (arXiv 2406.05128), and its
 * adjoint, batched over B independent signals:
 *
 *   forward   (Eq. 5)   s(t)  = e(t) - sum_{i=1..M} a_i(t) s(t-i)
 *   adjoint   (Eq. 11)  ge(t) = gs(t) - sum_{i=1..M} a_i(t+i) ge(t+i),
 *                       run from t = T-1 down to 0, ge(t >= T) = 0
 *   coeffs    (Eq. 12)  ga_i(t) = -ge(t) s(t-i)
 *   state     (extension of the zero initial conditions of Sec. 2.2)
 *                       s(-j) = zi[j-1];  gzi[j-1] = dL/ds(-j)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named a, e, s, ... are DEVICE pointers owned by the caller,
 *   row-major and densely packed:
 *     a      [B][T][M]   a[(b*T + t)*M + (i-1)] = a_i(t) of signal b
 *     e, s   [B][T]
 *     zi     [B][M]      zi[b*M + j-1] = s_b(-j); NULL means zero state
 *   _f32 entry points take float, _f64 entry points take double.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every call only enqueues work on that stream; none
 *   synchronises it.  Results are valid once the stream has reached the
 *   point of the call.
 * - `workspace` is caller-owned device memory of at least
 *   lp_tv_workspace_bytes(...) bytes, 256-byte aligned, for the same
 *   (B, T, M, chunk, dtype).  The library allocates no device memory.
 *   A workspace must not be used by two calls that may run concurrently.
 *   After lp_tv_forward it holds the chunk transfer matrices of `a`, which
 *   lp_tv_backward can reuse (LP_BWD_REUSE_FORWARD).
 * - `chunk` is the chunk length L of the parallel scan (samples).  0 asks
 *   the library to pick it (lp_tv_pick_chunk).  A non-zero value is rounded
 *   up to a multiple of 16.  Results depend on the chunk length only through
 *   floating-point rounding.
 * - No input may alias an output.
 * - Shapes: B >= 0, T >= 0, 0 <= M <= 32 (M <= 16 for _f64).  B == 0 or
 *   T == 0 is a no-op.  M == 0 copies e to s (and gs to ge).  M > T is
 *   allowed.
 * - Return value: LP_OK (0) or a negative error code; lp_strerror() names
 *   it.  An error is returned before any work is enqueued, except
 *   LP_ECUDA, which reports a failed launch (the stream may then hold part
 *   of the work).  Errors never abort the process.
 */
#ifndef TVLP_H
#define TVLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LP_OK = 0,
    LP_EINVAL = -1,       /* bad shape, NULL required pointer, bad flag  */
    LP_EUNSUPPORTED = -2, /* order M beyond what this build supports     */
    LP_EWORKSPACE = -3,   /* workspace NULL, too small or misaligned      */
    LP_ECUDA = -4,        /* a CUDA launch or runtime call failed         */
    LP_EALIGN = -5,       /* a data pointer is not aligned to its type    */
    LP_ETOOBIG = -6,      /* problem too large for the fixed scratch      */
    LP_ETIMEOUT = -7,     /* a bounded host-side wait ended first         */
    LP_ENONFINITE = -8    /* lp_tv_check_finite_*: an inf or NaN found    */
};

enum { LP_DTYPE_F32 = 0, LP_DTYPE_F64 = 1 };

/* lp_tv_backward flags. */
enum {
    /* The workspace still holds what lp_tv_forward left in it for the same
     * a, B, T, M, chunk and dtype: the chunk transfer matrices of the
     * forward.  The adjoint's chunk transfer is their transpose (the
     * adjoint state is the gradient with respect to the forward state), so
     * the backward then runs one recursion per chunk instead of M+1. */
    LP_BWD_REUSE_FORWARD = 1,
    /* The chunked adjoint re-run writes ga as it produces ge (one kernel
     * and one pass over the rows instead of two), when M is one of the
     * compiled orders; otherwise ga comes from a pass of its own over ge and
     * s.  Both give the same bits.  At B=32, T=48000, M=22 on a GB300 the
     * fused re-run takes 65 us against 32 + 27 us for the two kernels: its
     * gradient rows leave through the same two-stage shared ring that
     * prefetches the coefficients, which then runs shallower. */
    LP_BWD_FUSED_GA = 2
};

/* Which kernels compute the recursion. */
enum {
    LP_ALGO_CHUNKED = 0, /* chunked parallel scan (default, fast path)  */
    LP_ALGO_PLAIN = 1    /* one thread per signal, sequential in time   */
};

/*
 * Non-finite check: one pass over x [n] (DEVICE memory) on `stream`.
 * Returns LP_ENONFINITE if any element is an infinity or NaN, LP_OK if
 * none is (or n == 0), LP_EINVAL for x NULL with n > 0, LP_EALIGN for x
 * not aligned to its type.  The recursions carry a non-finite value to every
 * later sample of its signal, and a filter with a pole outside the unit
 * circle overflows FP32 to inf (the literal |k| <= 0.95 generator at M=22
 * does so in long signals).  So a caller checks a, e, gs before a call,
 * and s, ge, ga after one, when its inputs are not known to be finite and
 * stable.  The call synchronises `stream` (it reads the result back) and
 * so cannot be captured in a graph.  Up to 64 checks may run at once from
 * different threads or streams.
 */
int lp_tv_check_finite_f32(const float *x, size_t n, void *stream);
int lp_tv_check_finite_f64(const double *x, size_t n, void *stream);

/*
 * Per-kernel timing hook.  `events` points to 2*n cudaEvent_t handles
 * (passed as void*) created by the caller.  While installed, every later
 * forward/backward call made from the calling thread records events[2k]
 * just before and events[2k+1] just after its k-th kernel launch (k < n) on
 * the call's stream.  Kernel order: forward (chunked) summary, scan,
 * re-run; backward (chunked) zero-state summary (or full summary without
 * LP_BWD_REUSE_FORWARD), scan, re-run, coefficient gradient (none when the
 * re-run writes ga itself, see LP_BWD_FUSED_GA; for the
 * generated-coefficient calls: gradient, then its final sum); the plain
 * algorithm launches re-run (and coefficient gradient).  NULL uninstalls the
 * hook.  The library neither creates nor destroys events.
 */
int lp_tv_set_profile_events(void **events, int n);

/*
 * Threads per signal of the chunked FP32 calls with streamed coefficients
 * (uniform and varlen batches; the choice an autotuner makes beside the
 * chunk length, no counterpart in the paper).  Applies to the later calls
 * made from the calling thread:
 *   k1_lane_factor       1: the summary pass runs a chunk's M+1 recursions
 *                        on G lanes (the default packing for the order),
 *                        2: on 2G lanes with half the recursions each;
 *   rerun_chunks_per_warp  16 (default) or 8 chunks per warp in the
 *                        one-recursion passes.
 * 0 selects the default.  Results are the same up to floating-point
 * rounding (the packing changes the order of the summary's operations).
 * LP_EINVAL for other values.  Mixed-order calls keep their own shapes.
 */
int lp_tv_set_threads_per_chunk(int k1_lane_factor, int rerun_chunks_per_warp);

/* Human-readable name of an error code. Never NULL. */
const char *lp_strerror(int code);

/* Library version string, e.g. "tvlp 0.1 sm_103a". */
const char *lp_version(void);

/* Chunk length the library picks for (B, T, M) when `chunk` is 0. */
int lp_tv_pick_chunk(int B, int64_t T, int M, int dtype);

/* Number of chunks per signal for (T, M, chunk) after rounding. */
int64_t lp_tv_num_chunks(int64_t T, int M, int chunk);

/*
 * Workspace bytes needed by lp_tv_forward_* / lp_tv_backward_* for the
 * given problem (scan summaries and chunk states).  Returns 0 for an
 * invalid shape.
 */
size_t lp_tv_workspace_bytes(int B, int64_t T, int M, int chunk, int dtype);

/*
 * Forward filter, Eq. 5 (Sec. 3.2), batched.
 *   a    [B][T][M]  coefficients a_i(t)                        (in)
 *   e    [B][T]     excitation                                  (in)
 *   zi   [B][M]     initial state s(-j) = zi[j-1], or NULL      (in)
 *   s    [B][T]     output                                      (out)
 *   ckpt [B][nC][M] incoming state of each chunk, or NULL       (out)
 *                   ckpt[(b*nC + c)*M + j-1] = s_b(c*L - j), nC =
 *                   lp_tv_num_chunks(T, M, chunk); these are the chunk
 *                   checkpoints the backward can recompute s from.
 *   algo            LP_ALGO_CHUNKED or LP_ALGO_PLAIN (ckpt requires CHUNKED)
 */
int lp_tv_forward_f32(int B, int64_t T, int M, const float *a, const float *e,
                      const float *zi, float *s, float *ckpt, int chunk,
                      int algo, void *workspace, size_t workspace_bytes,
                      void *stream);
int lp_tv_forward_f64(int B, int64_t T, int M, const double *a, const double *e,
                      const double *zi, double *s, double *ckpt, int chunk,
                      int algo, void *workspace, size_t workspace_bytes,
                      void *stream);

/*
 * Adjoint, Eqs. 11-12 (Sec. 3.2.1-3.2.2), batched.
 *   gs   [B][T]     upstream gradient dL/ds                     (in)
 *   a    [B][T][M]  coefficients used by the forward            (in)
 *   s    [B][T]     forward output (needed for ga)              (in)
 *   zi   [B][M]     forward initial state or NULL               (in)
 *   ge   [B][T]     dL/de                                       (out)
 *   ga   [B][T][M]  dL/da_i(t) = -ge(t) s(t-i), or NULL         (out)
 *   gzi  [B][M]     dL/ds(-j), or NULL                          (out)
 *   flags           0, LP_BWD_REUSE_FORWARD, LP_BWD_FUSED_GA (or both)
 * `s` may be NULL only when `ga` is NULL.
 */
int lp_tv_backward_f32(int B, int64_t T, int M, const float *gs, const float *a,
                       const float *s, const float *zi, float *ge, float *ga,
                       float *gzi, int chunk, int algo, int flags,
                       void *workspace, size_t workspace_bytes, void *stream);
int lp_tv_backward_f64(int B, int64_t T, int M, const double *gs,
                       const double *a, const double *s, const double *zi,
                       double *ge, double *ga, double *gzi, int chunk, int algo,
                       int flags, void *workspace, size_t workspace_bytes,
                       void *stream);

/*
 * Adjoint from chunk checkpoints (chunk-state checkpointing, a memory
 * saving with no counterpart in the paper): instead of the forward output
 * s, the caller keeps the per-chunk incoming states `ckpt` that
 * lp_tv_forward_* wrote (with the same `chunk`) and the excitation e.  The
 * call first re-runs the forward pass of every chunk from its checkpoint
 * into the caller's buffer `s` (bit for bit what the forward wrote), then
 * computes ge, ga, gzi as lp_tv_backward_* with the chunked algorithm.
 *   e    [B][T]     excitation of the forward                   (in)
 *   ckpt [B][nC][M] incoming state of every chunk, from the forward (in)
 *   s    [B][T]     scratch, holds the recomputed forward output  (out)
 * Other arguments as lp_tv_backward_*; `flags` may hold
 * LP_BWD_REUSE_FORWARD (when the workspace still holds that forward's maps)
 * and LP_BWD_FUSED_GA.
 * Memory kept between forward and backward is ckpt (M values per chunk:
 * 0.55 B/sample at M=22, chunk 160) instead of s (4 B/sample).
 */
int lp_tv_backward_recompute_f32(int B, int64_t T, int M, const float *gs,
                                 const float *a, const float *e,
                                 const float *ckpt, const float *zi, float *s,
                                 float *ge, float *ga, float *gzi, int chunk,
                                 int flags, void *workspace,
                                 size_t workspace_bytes, void *stream);
int lp_tv_backward_recompute_f64(int B, int64_t T, int M, const double *gs,
                                 const double *a, const double *e,
                                 const double *ckpt, const double *zi,
                                 double *s, double *ge, double *ga,
                                 double *gzi, int chunk, int flags,
                                 void *workspace, size_t workspace_bytes,
                                 void *stream);

/*
 * Varlen batches (uneven batching of signals; no counterpart in the
 * paper): n signals of different lengths packed back to back, one call.
 *   offsets [n+1]   DEVICE array, int64: signal b holds rows
 *                   [offsets[b], offsets[b+1]); offsets[0] = 0,
 *                   non-decreasing; `total` = offsets[n] (passed on the host
 *                   for sizing).  A signal may be empty.
 *   a [total][M], e / s / gs / ge [total], ga [total][M]  packed rows
 *   zi / gzi [n][M]  per signal (NULL: zero state)
 *   ckpt [nQ][M]     incoming state of every chunk, signals in order, each
 *                    signal's chunks in order; nQ = sum_b ceil(len_b / L)
 * Every signal is cut into chunks of `chunk` rows (0: picked from n and
 * total/n; rounded up to a multiple of 16) from its own start, and its scan
 * groups depend only on its own chunk count, so with a fixed `chunk` a
 * signal's results do not depend on the rest of the batch (bit for bit).
 * Coefficient rows start 16-byte aligned when offsets are even; odd offsets
 * work but load through a slower path.  Algorithm: chunked only.  Returns
 * and errors as the uniform calls; the workspace comes from
 * lp_tv_workspace_bytes_varlen with the same (n, total, M, chunk, dtype).
 */
size_t lp_tv_workspace_bytes_varlen(int n, int64_t total, int M, int chunk,
                                    int dtype);
int lp_tv_forward_varlen_f32(int n, const int64_t *offsets, int64_t total,
                             int M, const float *a, const float *e,
                             const float *zi, float *s, float *ckpt,
                             int chunk, void *workspace,
                             size_t workspace_bytes, void *stream);
int lp_tv_forward_varlen_f64(int n, const int64_t *offsets, int64_t total,
                             int M, const double *a, const double *e,
                             const double *zi, double *s, double *ckpt,
                             int chunk, void *workspace,
                             size_t workspace_bytes, void *stream);
int lp_tv_backward_varlen_f32(int n, const int64_t *offsets, int64_t total,
                              int M, const float *gs, const float *a,
                              const float *s, const float *zi, float *ge,
                              float *ga, float *gzi, int chunk, int flags,
                              void *workspace, size_t workspace_bytes,
                              void *stream);
int lp_tv_backward_varlen_f64(int n, const int64_t *offsets, int64_t total,
                              int M, const double *gs, const double *a,
                              const double *s, const double *zi, double *ge,
                              double *ga, double *gzi, int chunk, int flags,
                              void *workspace, size_t workspace_bytes,
                              void *stream);

/*
 * Mixed orders (uneven batching of signals of different lengths AND orders
 * in one call; no counterpart in the paper, whose Eq. 5 fixes one order per
 * filter): signal b has len_b = offsets[b+1] - offsets[b] samples and its
 * own order M_b = orders[b], 1 <= M_b <= 32.  Each call runs one launch per
 * kernel role over the whole batch: signals are grouped by the padded order
 * the kernels are compiled for (2, 4, 8, 12, 16, 22, 30, 32), and each block
 * of a launch runs the code of its group's order; a signal keeps its own
 * order inside its group.
 *   offsets [n+1]  DEVICE, int64: rows of signal b in e, s, gs, ge are
 *                  [offsets[b], offsets[b+1]); offsets[0] = 0, non-decreasing
 *   orders  [n]    DEVICE, int32
 *   offsets_host, orders_host: the same arrays in HOST memory (the library
 *                  plans the groups, grids and workspace from them)
 *   a, ga          coefficients of signal b: len_b rows of M_b values,
 *                  row-major, starting at element aoff[b] with aoff[0] = 0
 *                  and aoff[b+1] = aoff[b] + len_b*M_b rounded up to a
 *                  multiple of 4 (so every block starts 16-byte aligned);
 *                  lp_tv_mixed_coeff_offsets writes aoff [n+1] (HOST) and
 *                  returns the total element count
 *   zi, gzi [n][32] initial state: zi[b*32 + j-1] = s_b(-j), j <= M_b
 *                  (NULL: zero state)
 * `chunk` 0 picks each group's chunk length from its signal count and
 * lengths; with a fixed chunk a signal's results do not depend on the rest
 * of the batch (bit for bit), and equal those of a single-order varlen call
 * with that chunk.  The chunked algorithm with the defect correction, as for
 * the other FP32 calls; no checkpoints and no LP_BWD_FUSED_GA.  Workspace:
 * lp_tv_workspace_bytes_mixed (0 for invalid arguments).  Errors as for
 * the varlen calls; an order outside 1..32 gives LP_EINVAL or
 * LP_EUNSUPPORTED.  A backward with LP_BWD_REUSE_FORWARD must get the
 * forward's workspace, chunk, offsets and orders.
 */
int64_t lp_tv_mixed_coeff_offsets(int n, const int64_t *offsets_host,
                                  const int *orders_host, int64_t *aoff_host);
size_t lp_tv_workspace_bytes_mixed(int n, const int64_t *offsets_host,
                                   const int *orders_host, int chunk);
int lp_tv_forward_mixed_f32(int n, const int64_t *offsets, const int *orders,
                            const int64_t *offsets_host,
                            const int *orders_host, const float *a,
                            const float *e, const float *zi, float *s,
                            int chunk, void *workspace, size_t workspace_bytes,
                            void *stream);
int lp_tv_backward_mixed_f32(int n, const int64_t *offsets, const int *orders,
                             const int64_t *offsets_host,
                             const int *orders_host, const float *gs,
                             const float *a, const float *s, const float *zi,
                             float *ge, float *ga, float *gzi, int chunk,
                             int flags, void *workspace,
                             size_t workspace_bytes, void *stream);

/*
 * Coefficients generated in the kernels instead of streamed (FP32, chunked
 * algorithm; the per-sample coefficient preparation of Sec. 4.3 and the
 * time-invariant filter of Sec. 2.2 / Eq. 2).  Every pass that would read
 * a row a(t) computes it from a small input instead:
 *
 * Frames: k [B][F][M] reflection coefficients per frame, F = ceil(T/hop)+1,
 *   k[(b*F + f)*M + m-1] = k_m of frame f of signal b.  Frame f is anchored
 *   at sample f*hop and linearly interpolated to every sample,
 *     k_m(t) = k_m[f] + w (k_m[f+1] - k_m[f]),  f = t / hop,
 *     w = (t - f*hop) / hop,
 *   then stepped up to the direct form of A(z) = 1 + sum_i a_i z^-i:
 *     a^(m)_i = a^(m-1)_i + k_m a^(m-1)_{m-i} (i < m),  a^(m)_m = k_m,
 *   and a(t) = a^(M).  The filter is Eq. 5 with that a(t).  The backward
 *   returns ge (Eq. 11), gzi, and gk [B][F][M] = dL/dk: Eq. 12 taken
 *   through the step-up and the interpolation (NULL: not computed).
 * Time-invariant: a [B][M], one coefficient row per signal (Eq. 2).  The
 *   backward returns ga [B][M] = sum_t dL/da(t) (Eq. 12 summed over time,
 *   which is Eq. 3's two-filter gradient).
 * Workspace: lp_tv_workspace_bytes_frames / _ti (the scan's workspace plus
 * the gradient's scratch).  A forward leaves the chunk transfers in it for
 * a backward with LP_BWD_REUSE_FORWARD, as for the streamed calls.  Other
 * conventions, shapes and errors as for lp_tv_forward_f32 /
 * lp_tv_backward_f32; hop >= 1.
 *
 * Row cache (frames, uniform batches): with a workspace of at least
 * lp_tv_workspace_bytes_frames_cached bytes and M one of the compiled
 * orders (2, 4, 8, 12, 16, 22, 30, 32), the forward's first pass also
 * writes every generated row a(t) into the workspace (4*M bytes per
 * sample), and its re-run streams them instead of generating them again.
 * A backward with LP_BWD_REUSE_FORWARD on that workspace streams them too:
 * that flag promises the workspace still holds what the forward on the
 * same k left in it.  Results are the same bits either way.  For other M,
 * lp_tv_workspace_bytes_frames_cached equals lp_tv_workspace_bytes_frames.
 *
 * lp_tv_forward_frames_varlen_f32 / lp_tv_backward_frames_varlen_f32:
 * varlen batches (offsets as for lp_tv_forward_varlen_f32) with
 * frame_offsets [n] (DEVICE, int64): signal b's frames start at frame
 * frame_offsets[b] of k, and it has ceil(len_b/hop)+1 of them, len_b =
 * offsets[b+1] - offsets[b]; total_frames = the rows of k (and of gk).
 * Workspace: lp_tv_workspace_bytes_varlen for the forward (and a backward
 * without gk), lp_tv_workspace_bytes_frames_varlen for a backward with gk.
 * lp_tv_workspace_bytes_frames_varlen_cached adds the row cache described
 * above (4*M bytes per packed row, compiled orders): the varlen forward
 * keeps its generated rows in such a workspace, and a backward with
 * LP_BWD_REUSE_FORWARD on it streams them.  Where the cached rows start
 * depends on the chunk length and on workspace_bytes, and the backward
 * cannot tell whether the forward wrote them: a backward with
 * LP_BWD_REUSE_FORWARD must get the same workspace, workspace_bytes, chunk,
 * offsets, frame_offsets and k as the forward, or it reads stale rows.
 */
size_t lp_tv_workspace_bytes_frames(int B, int64_t T, int M, int hop,
                                    int chunk);
size_t lp_tv_workspace_bytes_frames_cached(int B, int64_t T, int M, int hop,
                                           int chunk);
int lp_tv_forward_frames_f32(int B, int64_t T, int M, int hop,
                             const float *k, const float *e,
                             const float *zi, float *s, float *ckpt,
                             int chunk, void *workspace,
                             size_t workspace_bytes, void *stream);
int lp_tv_backward_frames_f32(int B, int64_t T, int M, int hop,
                              const float *gs, const float *k,
                              const float *s, const float *zi, float *ge,
                              float *gk, float *gzi, int chunk, int flags,
                              void *workspace, size_t workspace_bytes,
                              void *stream);
int lp_tv_forward_frames_varlen_f32(int n, const int64_t *offsets,
                                    int64_t total, int M, int hop,
                                    const int64_t *frame_offsets,
                                    const float *k, const float *e,
                                    const float *zi, float *s, float *ckpt,
                                    int chunk, void *workspace,
                                    size_t workspace_bytes, void *stream);
size_t lp_tv_workspace_bytes_frames_varlen(int n, int64_t total, int M,
                                           int64_t total_frames, int chunk);
size_t lp_tv_workspace_bytes_frames_varlen_cached(int n, int64_t total, int M,
                                                  int64_t total_frames,
                                                  int chunk);
int lp_tv_backward_frames_varlen_f32(int n, const int64_t *offsets,
                                     int64_t total, int M, int hop,
                                     const int64_t *frame_offsets,
                                     int64_t total_frames, const float *gs,
                                     const float *k, const float *s,
                                     const float *zi, float *ge, float *gk,
                                     float *gzi, int chunk, int flags,
                                     void *workspace, size_t workspace_bytes,
                                     void *stream);
size_t lp_tv_workspace_bytes_ti(int B, int64_t T, int M, int chunk);
int lp_tv_forward_ti_f32(int B, int64_t T, int M, const float *a,
                         const float *e, const float *zi, float *s,
                         float *ckpt, int chunk, void *workspace,
                         size_t workspace_bytes, void *stream);
int lp_tv_backward_ti_f32(int B, int64_t T, int M, const float *gs,
                          const float *a, const float *s, const float *zi,
                          float *ge, float *ga, float *gzi, int chunk,
                          int flags, void *workspace,
                          size_t workspace_bytes, void *stream);

/*
 * Device status word of the current device: 0 while every bounded wait
 * inside the kernels completed, 1 once a shared-memory bulk-copy wait gave
 * up, 2 once a scan wait for other warps' results gave up (the kernel then
 * stopped early and its outputs are not valid).  In a library compiled with
 * TVLP_CHECK_BOUNDS (the checked build the tests use), 16 + n records that
 * index check n failed: a chunk, scan item or correction-list entry built on
 * the device lay outside the range it must lie in, and the work it guards
 * was skipped.  Reads it synchronously (waits for the device's outstanding
 * work) and clears it when `reset` is non-zero.  Returns the status or
 * LP_ECUDA.
 */
int lp_tv_device_status(int reset);

/*
 * L2 set-aside for the passes' evict-last stages (no counterpart in the
 * paper).  Consecutive passes over `a` mark the stages the next pass reads
 * first as evict-last (createpolicy L2::evict_last); the hardware keeps such
 * lines in the persisting part of L2, which is 0 bytes unless the process
 * sets it aside.  This sets the current context's persisting L2 size
 * (cudaLimitPersistingL2CacheSize) to `bytes`, clipped to the device's
 * maximum, and writes the size applied to *applied (may be NULL).  The
 * limit belongs to this process's context and ends with it.  LP_ECUDA if a
 * runtime call fails.
 */
int lp_tv_l2_set_aside(size_t bytes, size_t *applied);

/*
 * Failure-detection self-test (no counterpart in the paper).  Launches one
 * warp on `stream` that runs one of the kernels' bounded waits on a
 * condition nothing satisfies: which = 1, an mbarrier waiting for bulk-copy
 * bytes that are never sent (no copy is issued); which = 2, a progress
 * counter that nothing increments.  The wait gives up after the same limit
 * the kernels use (well under a second), records status 1 or 2 in the
 * device status word (lp_tv_device_status) and returns; the context stays
 * usable.  LP_EINVAL for another `which`, LP_ECUDA if the launch fails.
 */
int lp_tv_selftest_wait(int which, void *stream);

/*
 * Frame-wise overlap-add approximation (Sec. 3.2: the frame-wise LP of the
 * earlier GOLF work that the sample-wise filter replaces; Sec. 5.2: 75 %
 * overlap; Sec. 4.3: the training-speed comparison of GOLF-ss with GOLF-ff).
 * Not Eq. 5: every frame is filtered by a time-invariant filter (Eq. 2).
 *   Frames of N = 4*hop samples start every hop samples: frame f covers
 *   samples t_f .. t_f + N - 1, t_f = (f - 3)*hop, and there are
 *   F = lp_framewise_num_frames(T, hop) = ceil(T/hop) + 3 of them, so every
 *   sample lies in exactly four.  With w(n) = (1 - cos(2 pi n/N)) / 4 (the
 *   four windows over a sample sum to one):
 *     y_f(n) = w(n) e(t_f + n) - sum_{i=1..M} af_i y_f(n - i),  y_f(n<0) = 0
 *     s(t)   = sum_f y_f(t - t_f)   (e = 0 outside 0..T-1)
 *   The adjoint runs Eq. 11 with each frame's coefficients over the frame,
 *     gu_f(n) = gs(t_f + n) - sum_i af_i gu_f(n + i),  gu_f(n >= N) = 0,
 *     ge(t)   = sum_f w(t - t_f) gu_f(t - t_f),
 *     gaf_i   = -sum_n gu_f(n) y_f(n - i)    (Eq. 12 summed over the frame).
 * Arguments (DEVICE pointers, FP32, caller-owned):
 *   af   [B][F][M] direct-form coefficients of every frame           (in)
 *   e, s [B][T]    excitation (in) and output (out)
 *   y    [B][N][F] frame outputs y_f(n) at y[(b*N + n)*F + f], written by
 *                  the forward when not NULL, read by the backward;
 *                  lp_framewise_outputs_bytes(B, T, hop) bytes
 *   gs, ge [B][T]  dL/ds (in), dL/de (out); gaf [B][F][M] dL/daf (out)
 * hop: a multiple of 8, 8 <= hop <= 512; 0 <= M <= 32.  One kernel per
 * call, enqueued on `stream`; nothing is allocated.  Returns LP_OK,
 * LP_EINVAL (shape, hop or a required NULL pointer), LP_EUNSUPPORTED
 * (M > 32 or T >= 2^31) or LP_ECUDA.
 */
int64_t lp_framewise_num_frames(int64_t T, int hop);
size_t lp_framewise_outputs_bytes(int B, int64_t T, int hop);
int lp_framewise_forward_f32(int B, int64_t T, int M, int hop, const float *af,
                             const float *e, float *s, float *y, void *stream);
int lp_framewise_backward_f32(int B, int64_t T, int M, int hop,
                              const float *af, const float *y,
                              const float *gs, float *ge, float *gaf,
                              void *stream);

/*
 * Allocation-free forward filter (no counterpart in the paper; a service for
 * callers that cannot allocate device memory when they run the filter, such
 * as a real-time audio callback that must not wait on the CUDA allocator or
 * a plugin whose host application owns the GPU memory budget).
 *
 * Same arguments, layouts and results as lp_tv_forward_f32 with chunk = 0
 * and the chunked algorithm, but no workspace: the scan's scratch data live
 * in an array of LP_NOALLOC_SCRATCH_BYTES compiled into the library.  Every
 * GPU that loads the library holds that array until the process exits.
 * - Problems whose scratch (lp_tv_workspace_bytes(B, T, M, 0, LP_DTYPE_F32))
 *   exceeds LP_NOALLOC_SCRATCH_BYTES are rejected with LP_ETOOBIG before any
 *   work is enqueued; order limits are those of lp_tv_forward_f32.
 * - The call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 *   library routine.
 * - The first call on a device looks up the array's device address for that
 *   device; make that first call before any stream capture on the device.
 * - All calls share the one array, which keeps what the last call wrote:
 *   calls that may overlap on the GPU (different streams, no ordering
 *   between them) race on it and must be serialised by the caller.
 */
#define LP_NOALLOC_SCRATCH_BYTES (32u << 20)
int lp_tv_forward_noalloc_f32(int B, int64_t T, int M, const float *a,
                              const float *e, const float *zi, float *s,
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TVLP_H */
