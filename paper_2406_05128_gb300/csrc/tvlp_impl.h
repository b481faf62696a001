// Host-side declarations shared by the C ABI and the per-order kernel
// instantiations.  Each (scalar type, padded order MP) pair is compiled in
// its own translation unit (tvlp_inst.cu with -DTVLP_SCALAR/-DTVLP_MP) so the
// build runs in parallel.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tvlp {

// One batched problem after validation and chunk selection.
struct Problem {
    int B;        // signals
    int64_t T;    // samples per signal
    int M;        // real order (1..MP)
    int MP;       // padded order (template parameter of the kernels)
    int L;        // chunk length, a multiple of 16
    int64_t nC;   // chunks per signal
    int64_t NQ;   // B * nC
    int G2;       // chunks per group of the two-level scan
    int nG;       // groups per signal
    int64_t items;  // scan groups in the batch (varlen: an upper bound)
    // varlen batches (off != nullptr): signals packed back to back, signal b
    // at rows [off[b], off[b+1]) (device array, caller-owned); T is then the
    // total row count, nC unused and NQ an upper bound of the chunk count;
    // the prefix tables live in the workspace (region 8)
    const int64_t *off;
    int *status;  // device status word (bounded waits record timeouts here)
};

// Where the streamed passes take the coefficient rows a(t) from.
//   SRC_STREAM  read a [rows][M] from memory (the default path)
//   SRC_CONST   one row per signal, k = a [signals][M]: the time-invariant
//               filter of Eq. 2
//   SRC_FRAMES  generated in the kernels from frame-rate reflection
//               coefficients k [frames][M] (Sec. 4.3): frame f is anchored
//               at sample f*hop, linearly interpolated to every sample, then
//               stepped up to the direct form,
//                 a^(m)_i = a^(m-1)_i + k_m a^(m-1)_{m-i} (i < m), a^(m)_m = k_m
//               Signal b's frames start at frame foff[b] (varlen) or b*F.
enum { SRC_STREAM = 0, SRC_CONST = 1, SRC_FRAMES = 2 };
struct CoefSrc {
    int kind = SRC_STREAM;
    const float *k = nullptr;
    const int64_t *foff = nullptr;  // varlen: first frame of every signal (device)
    int64_t F = 0;                  // frames per signal (uniform batches)
    int hop = 0;
    float inv_hop = 0.f;
    // SRC_FRAMES, M == MP: the forward's summary pass also writes every
    // generated row here ([rows][MP], rows in the order of `a`), and the
    // later passes stream them instead of generating them again
    float *cache = nullptr;
};

// Per-instantiation geometry the host needs before launching.
struct Shape {
    int chunks_per_warp;   // K1 chunks held by one warp
    int warps_per_block;   // K1 block size / 32
    int per_step_cycles;   // rough K1 issue cost of one time step (chunk picker)
    size_t ws_per_chunk;   // workspace bytes per chunk (summaries + states)
};

template <typename S, int MP> struct Impl {
    static Shape shape();
    static int forward(const Problem &p, const S *a, const S *e, const S *zi, S *s, S *ckpt, int algo,
                       void *ws, cudaStream_t st);
    // s from the chunk checkpoints of a chunked forward (same chunk length)
    static int rerun(const Problem &p, const S *a, const S *e, const S *ckpt, const S *zi, S *s, void *ws,
                     cudaStream_t st);
    static int backward(const Problem &p, const S *gs, const S *a, const S *s, const S *zi, S *ge, S *ga,
                        S *gzi, int algo, int flags, void *ws, cudaStream_t st);
    // The chunked forward and adjoint with the coefficient rows generated in
    // the kernels (src.kind SRC_CONST or SRC_FRAMES; FP32 only).  The
    // adjoint writes ge and gzi; the coefficient gradient is grad_src.
    static int forward_gen(const Problem &p, const CoefSrc &src, const S *e, const S *zi, S *s, S *ckpt, void *ws,
                           cudaStream_t st);
    static int backward_gen(const Problem &p, const CoefSrc &src, const S *gs, const S *s, const S *zi, S *ge,
                            S *gzi, int flags, void *ws, cudaStream_t st);
    // dL/d(source): SRC_CONST, gk [signals][M] = sum_t dL/da(t) (Eq. 12
    // summed over time, Eq. 3); SRC_FRAMES, gk [frames][M] through the
    // step-up and the interpolation.  `scratch` holds grad_src_scratch bytes.
    static int grad_src(const Problem &p, const CoefSrc &src, const S *ge, const S *s, const S *zi, S *gk,
                        void *scratch, cudaStream_t st);
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Status codes (mirror include/tvlp.h).
enum { OK = 0, EINVAL_ = -1, EUNSUPPORTED = -2, EWORKSPACE = -3, ECUDA = -4, EALIGN = -5 };
enum { ALGO_CHUNKED = 0, ALGO_PLAIN = 1 };
enum { BWD_REUSE_FORWARD = 1, BWD_FUSED_GA = 2 };

// Workspace regions (each 256-byte aligned), in elements of the scalar
// (RS = MP padded to 16 bytes, YS = (MP+1)*RS, ZS = RS):
//   0 Y  [NQ][YS]     chunk maps (forward; the adjoint's own when it
//                     cannot reuse the forward's)
//   1 X  [NQ][MP]     forward incoming state of every chunk
//   2 Z  [NQ][ZS]     adjoint zero-state summaries
//   3 W  [NQ][MP]     adjoint incoming state of every chunk
//   4 GY [B*nG][YS]   group maps of the two-level scan
//   5 GZ [B*nG][ZS]   adjoint group zero-state summaries
//   6 GX [B*nG][ZS]   incoming state of every group
//   7 CNT [B+1][32]   scan progress per signal (unsigned, one 128-byte
//                     line each), zeroed by the kernel before each scan
//   8 TAB [2][B+1]    varlen: first chunk and first scan group of every
//                     signal (int), built at the start of each call
//   9 LIST [NQ]       defect correction: the chunks pass 2 re-runs (int);
//                     their count is word 0 of a counter line after the
//                     signals' (CNT holds B+1 lines)
// Group regions hold p.items rows.
inline size_t rs_elems(int MP, size_t sz) { return (((size_t)MP * sz + 15) / 16) * 16 / sz; }
inline size_t ys_elems(int MP, size_t sz) { return (size_t)(MP + 1) * rs_elems(MP, sz); }
inline size_t zs_elems(int MP, size_t sz) { return rs_elems(MP, sz); }
inline size_t ws_offset(const Problem &p, size_t sz, int region) {
    const size_t items = (size_t)p.items;
    const size_t tab = p.off != nullptr ? 2 * ((size_t)p.B + 1) * sizeof(int) : 0;
    const size_t rows[10] = {(size_t)p.NQ * ys_elems(p.MP, sz),     (size_t)p.NQ * p.MP,
                             (size_t)p.NQ * zs_elems(p.MP, sz),     (size_t)p.NQ * p.MP,
                             items * ys_elems(p.MP, sz),            items * zs_elems(p.MP, sz),
                             items * zs_elems(p.MP, sz),            (((size_t)p.B + 1) * 32 * sizeof(unsigned) + sz - 1) / sz,
                             (tab + sz - 1) / sz,                   ((size_t)p.NQ * sizeof(int) + sz - 1) / sz};
    size_t off = 0;
    for (int r = 0; r < region; ++r) off += align256(rows[r] * sz);
    return off;
}
inline size_t ws_bytes(const Problem &p, size_t sz) { return ws_offset(p, sz, 10); }

// Threads per signal of the streamed FP32 calls made from this thread
// (lp_tv_set_threads_per_chunk): the summary pass's lanes per chunk
// (1: the default packing, 2: twice the lanes) and the re-run passes'
// chunks per warp (16 or 8).
struct LaunchShape {
    int k1_lane_factor;
    int rec_chunks;
};
LaunchShape launch_shape();

// Records the caller's profiling event for kernel k (begin or end) when a
// hook is installed on this thread (lp_tv_set_profile_events).
void profile_mark(int k, bool end, cudaStream_t st);

// The device status word of the current device (nullptr if unavailable).
int *device_status_word();

}  // namespace tvlp
