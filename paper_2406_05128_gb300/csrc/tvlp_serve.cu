// Serving loop: continuous batching of time-varying LP filter requests on one
// GPU (the C ABI is declared and documented in tvlp_serve.h).
//
// A worker thread turns the planner's iterations (serve_plan.h) into work on
// three streams:
//   in    host-to-device copies of the iteration's inputs and tables
//   comp  the adaptation call pair, the synthesis call, and the kernel that
//         carries the synthesis filter states to the next iteration
//   out   device-to-host copies of the outputs
// linked by events, so that iteration i+1's copies in run while iteration
// i's kernels run and iteration i-1's results come back.  All kernels run on
// `comp` in iteration order, which is what lets every call share one
// workspace and lets a continuing block read the state its previous block
// left.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "serve_plan.h"
#include "tvlp.h"
#include "tvlp_serve.h"

namespace {

using namespace tvlp_serve;

int64_t steady_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// zi_next[r][j] = s(end_r - 1 - j): the filter state after the r-th
// continuing block, in the zi convention s(-j) = zi[j-1] of the next block
// (Eq. 5 continued across the block boundary).  Rows r >= n_cont (requests
// that start in the next iteration) get the zero state.
__global__ void k_carry_state(const float *__restrict__ s, const int64_t *__restrict__ off,
                              const int *__restrict__ cont, int n_cont, int M, int rows, float *__restrict__ zi_next) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * M) return;
    const int r = (int)(i / M), j = (int)(i % M);
    float v = 0.f;
    if (r < n_cont) {
        // a continuing block is a full block: an even number >= M of rows,
        // no padding, so it ends where the next call slot starts
        const int64_t end = off[cont[r] + 1];
        v = s[end - 1 - j];
    }
    zi_next[i] = v;
}

constexpr int kCarryThreads = 256;
constexpr int kMaxInflight = 16;
// varlen tables, summary, scan, re-run, correction scan, correction re-run
constexpr int kFwdKernels = 6;
// varlen tables, zero-state, scan, re-run, correction scan, correction
// re-run, coefficient gradient
constexpr int kBwdKernels = 7;

struct Rec {
    Request req;
    const float *a = nullptr, *e = nullptr, *gs = nullptr;
    float *s = nullptr, *ge = nullptr, *ga = nullptr;
    int64_t arrival_ns = 0;
};

struct Done {
    int64_t id, latency_ns;
    int status;
};

struct Iter {
    IterPlan plan;
    int slot = 0;
};

struct Server {
    lp_serve_config cfg{};
    int device = 0, chunk = 0;
    char *dev = nullptr;  // one allocation: workspace | states | ring
    uint64_t dev_bytes = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    float *zi[2] = {nullptr, nullptr};
    char *ring = nullptr;
    Planner *planner = nullptr;
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kMaxInflight] = {}, ev_comp[kMaxInflight] = {}, ev_out[kMaxInflight] = {};
    char *tab_host = nullptr;  // pinned: max_inflight table slots
    uint64_t tab_slot_bytes = 0;

    std::deque<Iter> inflight;  // worker only
    uint64_t iter_count = 0;    // worker only

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Rec *> submitted;
    std::deque<Done> done;
    bool stop = false;
    std::atomic<int> error{LP_OK};
    int64_t n_submitted = 0, n_completed = 0;
    lp_serve_stats st{};
    std::thread worker;
};

int fail(Server &S, int code) {
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.error.load() == LP_OK) S.error.store(code);
    S.st.error = S.error.load();
    return code;
}

#define SV_CUDA(x)                                          \
    do {                                                    \
        if ((x) != cudaSuccess) return fail(S, LP_ECUDA);   \
    } while (0)
#define SV_LP(x)                                            \
    do {                                                    \
        const int rc_ = (x);                                \
        if (rc_ != LP_OK) return fail(S, rc_);              \
    } while (0)

// Enqueue one planned iteration on the three streams.
int issue(Server &S, Iter &it) {
    const IterPlan &P = it.plan;
    const Layout &L = P.lay;
    const int M = S.cfg.M, slot = it.slot;
    const size_t rowb = (size_t)M * sizeof(float);
    char *base = S.ring + P.offset;
    const int nf = (int)P.fwd.size(), na = (int)P.adapt.size(), nc = (int)P.cont.size();

    // tables: packed row offsets of both calls, continuing block indexes
    char *tab = S.tab_host + (size_t)slot * S.tab_slot_bytes;
    int64_t *off_f = reinterpret_cast<int64_t *>(tab + (L.off_f - L.tab));
    int64_t *off_a = reinterpret_cast<int64_t *>(tab + (L.off_a - L.tab));
    int *cont = reinterpret_cast<int *>(tab + (L.cont - L.tab));
    for (int k = 0; k < nf; ++k) off_f[k] = P.fwd[k].pos;
    off_f[nf] = P.rows_f;
    for (int k = 0; k < na; ++k) off_a[k] = P.adapt[k].pos;
    off_a[na] = P.rows_a;
    for (int k = 0; k < nc; ++k) cont[k] = P.cont[k];
    const int hop = S.cfg.hop;
    if (hop > 0) {
        int64_t *foff = reinterpret_cast<int64_t *>(tab + (L.foff - L.tab));
        for (int k = 0; k < nf; ++k) foff[k] = P.fwd[k].fpos;
        int64_t *foff_a = reinterpret_cast<int64_t *>(tab + (L.foff_a - L.tab));
        for (int k = 0; k < na; ++k) foff_a[k] = P.adapt[k].fpos;
    }
    // a block's frames: it starts on a frame anchor (block_rows is a multiple
    // of hop), and a padded block may need one frame more than the request
    // has, which repeats the request's last frame
    auto put_frames = [&](uint64_t dst, const Block &b, const Rec *r) {
        if (b.rows <= 0) return true;
        const int64_t f0 = b.row0 / hop, need = frames_of(padded(b.rows), hop);
        const int64_t have = frames_of(r->req.T, hop) - f0;
        const int64_t n = need < have ? need : have;
        char *d = base + dst + (size_t)b.fpos * rowb;
        if (cudaMemcpyAsync(d, r->a + f0 * M, (size_t)n * rowb, cudaMemcpyHostToDevice, S.s_in) != cudaSuccess)
            return false;
        for (int64_t x = n; x < need; ++x)
            if (cudaMemcpyAsync(d + (size_t)x * rowb, r->a + (f0 + have - 1) * M, rowb, cudaMemcpyHostToDevice,
                                S.s_in) != cudaSuccess)
                return false;
        return true;
    };
    SV_CUDA(cudaMemcpyAsync(base + L.tab, tab, L.tab_bytes, cudaMemcpyHostToDevice, S.s_in));

    auto put = [&](uint64_t dst, int64_t pos, const float *src, int64_t rows, size_t bytes_per_row, bool pad) {
        char *d = base + dst + (size_t)pos * bytes_per_row;
        if (rows > 0 && cudaMemcpyAsync(d, src, (size_t)rows * bytes_per_row, cudaMemcpyHostToDevice, S.s_in) !=
                            cudaSuccess)
            return false;
        if (pad && (rows & 1) && cudaMemsetAsync(d + (size_t)rows * bytes_per_row, 0, bytes_per_row, S.s_in) !=
                                     cudaSuccess)
            return false;
        return true;
    };
    for (const Block &b : P.fwd) {
        const Rec *r = static_cast<const Rec *>(b.req->user);
        if (hop > 0) {
            if (!put_frames(L.a_f, b, r) || !put(L.e_f, b.pos, r->e + b.row0, b.rows, sizeof(float), true))
                return fail(S, LP_ECUDA);
            continue;
        }
        if (!put(L.a_f, b.pos, r->a + b.row0 * M, b.rows, rowb, true) ||
            !put(L.e_f, b.pos, r->e + b.row0, b.rows, sizeof(float), true))
            return fail(S, LP_ECUDA);
    }
    for (const Block &b : P.adapt) {
        const Rec *r = static_cast<const Rec *>(b.req->user);
        const bool coef = hop > 0 ? put_frames(L.a_a, b, r) : put(L.a_a, b.pos, r->a, b.rows, rowb, true);
        if (!coef || !put(L.e_a, b.pos, r->e, b.rows, sizeof(float), true) ||
            !put(L.gs_a, b.pos, r->gs, b.rows, sizeof(float), true))
            return fail(S, LP_ECUDA);
    }
    SV_CUDA(cudaEventRecord(S.ev_in[slot], S.s_in));

    SV_CUDA(cudaStreamWaitEvent(S.s_comp, S.ev_in[slot], 0));
    int launches = 0;
    if (na > 0) {
        auto *oa = reinterpret_cast<const int64_t *>(base + L.off_a);
        auto *a = reinterpret_cast<const float *>(base + L.a_a);
        auto *s = reinterpret_cast<float *>(base + L.s_a);
        auto *e = reinterpret_cast<const float *>(base + L.e_a);
        auto *gs = reinterpret_cast<const float *>(base + L.gs_a);
        auto *ge = reinterpret_cast<float *>(base + L.ge_a);
        auto *ga = reinterpret_cast<float *>(base + L.ga_a);
        if (hop > 0) {
            // frames: a_a holds k, ga_a receives dL/dk
            auto *fa = reinterpret_cast<const int64_t *>(base + L.foff_a);
            SV_LP(lp_tv_forward_frames_varlen_f32(na, oa, P.rows_a, M, hop, fa, a, e, nullptr, s, nullptr, S.chunk, S.ws,
                                                  S.ws_bytes, S.s_comp));
            SV_LP(lp_tv_backward_frames_varlen_f32(na, oa, P.rows_a, M, hop, fa, P.frames_a, gs, a, s, nullptr, ge, ga,
                                                   nullptr, S.chunk, LP_BWD_REUSE_FORWARD, S.ws, S.ws_bytes,
                                                   S.s_comp));
            launches += kFwdKernels + kBwdKernels + 1;
        } else {
            SV_LP(lp_tv_forward_varlen_f32(na, oa, P.rows_a, M, a, e, nullptr, s, nullptr, S.chunk, S.ws, S.ws_bytes,
                                           S.s_comp));
            SV_LP(lp_tv_backward_varlen_f32(na, oa, P.rows_a, M, gs, a, s, nullptr, ge, ga, nullptr, S.chunk,
                                            LP_BWD_REUSE_FORWARD, S.ws, S.ws_bytes, S.s_comp));
            launches += kFwdKernels + kBwdKernels;
        }
    }
    const uint64_t it_no = S.iter_count;
    float *zi_cur = S.zi[it_no & 1], *zi_next = S.zi[(it_no + 1) & 1];
    if (nf > 0 && hop > 0) {
        SV_LP(lp_tv_forward_frames_varlen_f32(
            nf, reinterpret_cast<const int64_t *>(base + L.off_f), P.rows_f, M, hop,
            reinterpret_cast<const int64_t *>(base + L.foff), reinterpret_cast<const float *>(base + L.a_f),
            reinterpret_cast<const float *>(base + L.e_f), zi_cur, reinterpret_cast<float *>(base + L.s_f), nullptr,
            S.chunk, S.ws, S.ws_bytes, S.s_comp));
        launches += kFwdKernels;
    } else if (nf > 0) {
        SV_LP(lp_tv_forward_varlen_f32(nf, reinterpret_cast<const int64_t *>(base + L.off_f), P.rows_f, M,
                                       reinterpret_cast<const float *>(base + L.a_f),
                                       reinterpret_cast<const float *>(base + L.e_f), zi_cur,
                                       reinterpret_cast<float *>(base + L.s_f), nullptr, S.chunk, S.ws, S.ws_bytes,
                                       S.s_comp));
        launches += kFwdKernels;
    }
    {
        // the next iteration's states: carried rows first, zero after (also
        // when this iteration has no synthesis call)
        const int rows = S.cfg.max_signals;
        const int64_t n = (int64_t)rows * M;
        const unsigned grid = (unsigned)((n + kCarryThreads - 1) / kCarryThreads);
        k_carry_state<<<grid, kCarryThreads, 0, S.s_comp>>>(
            nf > 0 ? reinterpret_cast<const float *>(base + L.s_f) : nullptr,
            reinterpret_cast<const int64_t *>(base + L.off_f), reinterpret_cast<const int *>(base + L.cont), nc, M,
            rows, zi_next);
        SV_CUDA(cudaGetLastError());
        launches += 1;
    }
    SV_CUDA(cudaEventRecord(S.ev_comp[slot], S.s_comp));

    SV_CUDA(cudaStreamWaitEvent(S.s_out, S.ev_comp[slot], 0));
    auto get = [&](float *dst, uint64_t src, int64_t pos, int64_t rows, size_t bytes_per_row) {
        if (rows <= 0) return true;
        return cudaMemcpyAsync(dst, base + src + (size_t)pos * bytes_per_row, (size_t)rows * bytes_per_row,
                               cudaMemcpyDeviceToHost, S.s_out) == cudaSuccess;
    };
    for (const Block &b : P.fwd) {
        const Rec *r = static_cast<const Rec *>(b.req->user);
        if (!get(r->s + b.row0, L.s_f, b.pos, b.rows, sizeof(float))) return fail(S, LP_ECUDA);
    }
    for (const Block &b : P.adapt) {
        const Rec *r = static_cast<const Rec *>(b.req->user);
        // dL/da rows, or in frames mode dL/dk for the request's own frames
        const bool coef = hop > 0 ? (r->ga == nullptr || get(r->ga, L.ga_a, b.fpos, frames_of(r->req.T, hop), rowb))
                                  : get(r->ga, L.ga_a, b.pos, b.rows, rowb);
        if (!get(r->s, L.s_a, b.pos, b.rows, sizeof(float)) || !get(r->ge, L.ge_a, b.pos, b.rows, sizeof(float)) ||
            !coef)
            return fail(S, LP_ECUDA);
    }
    SV_CUDA(cudaEventRecord(S.ev_out[slot], S.s_out));

    std::lock_guard<std::mutex> lk(S.mu);
    lp_serve_stats &st = S.st;
    st.iterations += 1;
    st.synth_calls += nf > 0;
    st.adapt_calls += na > 0;
    st.kernel_launches += launches;
    st.blocks += nf;
    st.carried_blocks += P.n_carried;
    for (const Block &b : P.fwd) st.rows += b.rows;
    for (const Block &b : P.adapt) st.rows += b.rows;
    st.max_signals_iter = std::max<int64_t>(st.max_signals_iter, nf + na);
    st.ring_peak = std::max<uint64_t>(st.ring_peak, S.planner->ring().in_use());
    if (!S.inflight.empty()) st.overlapped += 1;
    return LP_OK;
}

// The oldest iteration's copies back are complete: its finished requests
// are done and its region is free.
void retire(Server &S, int status) {
    Iter &it = S.inflight.front();
    const int64_t t = steady_ns();
    {
        std::lock_guard<std::mutex> lk(S.mu);
        auto finish = [&](const Block &b) {
            if (!b.last) return;
            Rec *r = static_cast<Rec *>(b.req->user);
            S.done.push_back({r->req.id, t - r->arrival_ns, status});
            S.n_completed += 1;
            S.st.completed = S.n_completed;
            delete r;
        };
        for (const Block &b : it.plan.fwd) finish(b);
        for (const Block &b : it.plan.adapt) finish(b);
    }
    S.planner->release_oldest();
    S.inflight.pop_front();
    S.cv_done.notify_all();
}

// After an error: once the streams have stopped touching the requests'
// buffers, every request still in the server completes with the error.
void abandon(Server &S) {
    const int err = S.error.load();
    cudaStreamSynchronize(S.s_in);
    cudaStreamSynchronize(S.s_comp);
    cudaStreamSynchronize(S.s_out);
    while (!S.inflight.empty()) retire(S, err);
    IterPlan P;
    while (S.planner->plan(&P)) {
        S.inflight.push_back(Iter{P, 0});
        retire(S, err);
    }
}

void worker_main(Server *SP) {
    Server &S = *SP;
    if (cudaSetDevice(S.device) != cudaSuccess) fail(S, LP_ECUDA);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S.mu);
            if (S.inflight.empty() && !S.planner->has_work() && S.submitted.empty()) {
                if (S.stop) break;
                S.cv_work.wait(lk, [&] { return S.stop || !S.submitted.empty(); });
            }
            while (!S.submitted.empty()) {
                S.planner->enqueue(&S.submitted.front()->req);
                S.submitted.pop_front();
            }
            S.st.max_waiting = std::max<int64_t>(S.st.max_waiting, (int64_t)S.planner->waiting());
        }
        if (S.error != LP_OK) {
            abandon(S);
            continue;
        }
        bool progress = false;
        while (!S.inflight.empty()) {
            const cudaError_t q = cudaEventQuery(S.ev_out[S.inflight.front().slot]);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) {
                fail(S, LP_ECUDA);
                break;
            }
            retire(S, LP_OK);
            progress = true;
        }
        if (S.error != LP_OK) continue;
        if ((int)S.inflight.size() < S.cfg.max_inflight && S.planner->has_work()) {
            Iter it;
            if (S.planner->plan(&it.plan)) {
                it.slot = (int)(S.iter_count % (uint64_t)S.cfg.max_inflight);
                const int rc = issue(S, it);
                S.inflight.push_back(std::move(it));
                S.iter_count += 1;
                if (rc != LP_OK) continue;
                progress = true;
            }
        }
        if (!progress) std::this_thread::yield();
    }
}

void destroy_resources(Server *S) {
    for (int k = 0; k < kMaxInflight; ++k) {
        if (S->ev_in[k]) cudaEventDestroy(S->ev_in[k]);
        if (S->ev_comp[k]) cudaEventDestroy(S->ev_comp[k]);
        if (S->ev_out[k]) cudaEventDestroy(S->ev_out[k]);
    }
    if (S->s_in) cudaStreamDestroy(S->s_in);
    if (S->s_comp) cudaStreamDestroy(S->s_comp);
    if (S->s_out) cudaStreamDestroy(S->s_out);
    if (S->tab_host) cudaFreeHost(S->tab_host);
    if (S->dev) cudaFree(S->dev);
    delete S->planner;
    delete S;
}

}  // namespace

extern "C" {

void lp_serve_default_config(lp_serve_config *c) {
    if (c == nullptr) return;
    c->M = 22;
    c->chunk = 0;
    c->block_rows = 96000;
    c->max_signals = 256;
    c->max_iter_rows = int64_t(4) << 20;
    c->max_inflight = 4;
    c->hbm_budget = uint64_t(20) << 30;
    c->hop = 0;
}

int64_t lp_serve_now_ns(void) { return steady_ns(); }

int lp_serve_create(const lp_serve_config *cfg, void **server) {
    if (cfg == nullptr || server == nullptr) return LP_EINVAL;
    *server = nullptr;
    lp_serve_config c = *cfg;
    if (c.M < 1 || c.M > 32 || c.chunk < 0 || c.block_rows < 0 || c.max_signals < 1 || c.max_iter_rows < 2 ||
        c.max_inflight < 1 || c.max_inflight > kMaxInflight)
        return LP_EINVAL;
    if (c.hop < 0) return LP_EINVAL;
    if (c.block_rows > 0) {
        c.block_rows = std::max<int64_t>(padded(c.block_rows), padded(c.M));
        if (c.hop > 0) {
            // blocks start on frame anchors: a multiple of hop (and even)
            const int64_t q = c.hop % 2 == 0 ? c.hop : 2 * (int64_t)c.hop;
            c.block_rows = (c.block_rows + q - 1) / q * q;
        }
        if (c.block_rows > c.max_iter_rows) return LP_EINVAL;
    }
    int chunk = c.chunk;
    if (chunk == 0) {
        const int64_t typical = c.block_rows > 0 ? c.block_rows : 96000;
        chunk = lp_tv_pick_chunk(8, typical, c.M, LP_DTYPE_F32);
        if (chunk <= 0) return LP_EUNSUPPORTED;
    }
    chunk = (chunk + 15) / 16 * 16;

    // frames mode: the adaptation call's dL/dk scratch too; a call's frame
    // rows are at most rows/hop plus two per signal
    const int64_t max_frames = c.hop > 0 ? c.max_iter_rows / c.hop + 2 * (int64_t)c.max_signals + 2 : 0;
    const size_t ws = c.hop > 0 ? lp_tv_workspace_bytes_frames_varlen(c.max_signals, c.max_iter_rows, c.M, max_frames,
                                                                      chunk)
                                : lp_tv_workspace_bytes_varlen(c.max_signals, c.max_iter_rows, c.M, chunk, LP_DTYPE_F32);
    if (ws == 0) return LP_EUNSUPPORTED;
    const uint64_t ws_b = align256(ws), zi_b = align256((uint64_t)c.max_signals * c.M * sizeof(float));
    PlanConfig pc;
    pc.M = c.M;
    pc.block_rows = c.block_rows;
    pc.max_signals = c.max_signals;
    pc.max_iter_rows = c.max_iter_rows;
    pc.hop = c.hop;
    const uint64_t fixed = ws_b + 2 * zi_b;
    if (c.hbm_budget <= fixed) return LP_ETOOBIG;
    pc.ring_bytes = (c.hbm_budget - fixed) & ~uint64_t(255);
    if (pc.ring_bytes < max_region_bytes(pc)) return LP_ETOOBIG;

    Server *S = new (std::nothrow) Server();
    if (S == nullptr) return LP_ECUDA;
    S->cfg = c;
    S->chunk = chunk;
    S->planner = new Planner(pc);
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        destroy_resources(S);
        return LP_ECUDA;
    }
    S->dev_bytes = fixed + pc.ring_bytes;
    S->tab_slot_bytes = align256((uint64_t)(4 * c.max_signals + 2) * 8 + (uint64_t)c.max_signals * 4);
    bool ok = cudaMalloc(&S->dev, S->dev_bytes) == cudaSuccess;
    ok = ok && cudaHostAlloc(&S->tab_host, S->tab_slot_bytes * c.max_inflight, cudaHostAllocDefault) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&S->s_in, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&S->s_comp, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&S->s_out, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k < c.max_inflight; ++k) {
        ok = cudaEventCreateWithFlags(&S->ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->ev_comp[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->ev_out[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok) {
        S->ws = S->dev;
        S->ws_bytes = ws_b;
        S->zi[0] = reinterpret_cast<float *>(S->dev + ws_b);
        S->zi[1] = reinterpret_cast<float *>(S->dev + ws_b + zi_b);
        S->ring = S->dev + fixed;
        ok = cudaMemsetAsync(S->zi[0], 0, 2 * zi_b, S->s_comp) == cudaSuccess &&
             cudaStreamSynchronize(S->s_comp) == cudaSuccess;
    }
    if (!ok) {
        destroy_resources(S);
        return LP_ECUDA;
    }
    S->st.device_bytes = S->dev_bytes;
    S->st.ring_bytes = pc.ring_bytes;
    S->st.chunk = chunk;
    S->worker = std::thread(worker_main, S);
    *server = S;
    return LP_OK;
}

int lp_serve_submit(void *server, int64_t id, int kind, int64_t T, const float *a, const float *e, const float *gs,
                    float *s, float *ge, float *ga, int64_t arrival_ns) {
    Server *S = static_cast<Server *>(server);
    if (S == nullptr || T < 0 || (kind != LP_SERVE_SYNTH && kind != LP_SERVE_ADAPT)) return LP_EINVAL;
    if (T > 0 && (a == nullptr || e == nullptr || s == nullptr)) return LP_EINVAL;
    if (T > 0 && kind == LP_SERVE_ADAPT && (gs == nullptr || ge == nullptr || ga == nullptr)) return LP_EINVAL;
    if (!S->planner->admissible(kind, T)) return LP_ETOOBIG;
    Rec *r = new (std::nothrow) Rec();
    if (r == nullptr) return LP_ECUDA;
    r->req.id = id;
    r->req.T = T;
    r->req.kind = kind;
    r->req.user = r;
    r->a = a;
    r->e = e;
    r->gs = gs;
    r->s = s;
    r->ge = ge;
    r->ga = ga;
    r->arrival_ns = arrival_ns > 0 ? arrival_ns : steady_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->error != LP_OK) {
            delete r;
            return S->error.load();
        }
        S->submitted.push_back(r);
        S->n_submitted += 1;
        S->st.submitted = S->n_submitted;
    }
    S->cv_work.notify_one();
    return LP_OK;
}

int lp_serve_poll(void *server, int64_t *ids, int64_t *latency_ns, int *status, int max) {
    Server *S = static_cast<Server *>(server);
    if (S == nullptr || max < 0 || (max > 0 && (ids == nullptr || latency_ns == nullptr || status == nullptr)))
        return LP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    int n = 0;
    while (n < max && !S->done.empty()) {
        const Done &d = S->done.front();
        ids[n] = d.id;
        latency_ns[n] = d.latency_ns;
        status[n] = d.status;
        S->done.pop_front();
        ++n;
    }
    return n;
}

int lp_serve_drain(void *server, int64_t timeout_ms) {
    Server *S = static_cast<Server *>(server);
    if (S == nullptr) return LP_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto all_done = [&] { return S->n_completed == S->n_submitted; };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, all_done);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), all_done)) {
        return LP_ETIMEOUT;
    }
    return S->error.load();
}

int lp_serve_stats_get(void *server, lp_serve_stats *st, int reset) {
    Server *S = static_cast<Server *>(server);
    if (S == nullptr || st == nullptr) return LP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *st = S->st;
    if (reset) {
        lp_serve_stats &z = S->st;
        z.iterations = z.synth_calls = z.adapt_calls = z.kernel_launches = 0;
        z.blocks = z.carried_blocks = z.rows = z.max_signals_iter = z.max_waiting = z.overlapped = 0;
        z.ring_peak = 0;
    }
    return LP_OK;
}

int lp_serve_destroy(void *server) {
    Server *S = static_cast<Server *>(server);
    if (S == nullptr) return LP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    const int err = S->error.load();
    cudaStreamSynchronize(S->s_in);
    cudaStreamSynchronize(S->s_comp);
    cudaStreamSynchronize(S->s_out);
    destroy_resources(S);
    return err;
}

}  // extern "C"
