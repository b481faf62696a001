// CPU-only simulation of the serving loop's planner (serve_plan.h), built
// with the host compiler into libtvlp_plan.so so that the scheduling rules
// are tested without a GPU.  Time is counted in steps; one iteration is
// planned per step, and an iteration completes `lag` steps after it was
// planned (or earlier when nothing else can proceed), oldest first, which is
// the order in which the engine retires them.
#include <cstdint>
#include <deque>
#include <vector>

#include "serve_plan.h"

using namespace tvlp_serve;

extern "C" {

// Requests k = 0..n-1 arrive at step arrive[k] (non-decreasing), with length
// T[k] and kind kind[k]; hop > 0 plans a frames server.  Writes one row of 9
// int64 per block:
//   iteration, request, row0, rows, pos, call (0 synthesis, 1 adaptation),
//   carried, last, fpos (first frame row in the call, frames mode)
// and one row of 5 uint64 per iteration:
//   step planned, step completed, ring offset, region bytes, ring bytes in use
// Returns 0, -1 for bad arguments or a request no iteration can hold, -2
// when an output array is too small, -3 when the loop stopped making
// progress.
int lp_plan_simulate(int M, int64_t block_rows, int max_signals, int64_t max_iter_rows, uint64_t ring_bytes,
                     int hop, int lag, int n, const int64_t *T, const int *kind, const int64_t *arrive, int64_t cap_blocks,
                     int64_t *blocks, int64_t cap_iters, uint64_t *iters, int64_t *n_blocks, int64_t *n_iters) {
    if (M < 1 || max_signals < 1 || max_iter_rows < 2 || lag < 1 || n < 0 || n_blocks == nullptr ||
        n_iters == nullptr)
        return -1;
    PlanConfig c;
    c.M = M;
    c.block_rows = block_rows > 0 ? padded(block_rows) : 0;
    c.max_signals = max_signals;
    c.max_iter_rows = max_iter_rows;
    c.ring_bytes = ring_bytes;
    c.hop = hop;
    Planner P(c);
    std::vector<Request> req((size_t)n);
    for (int k = 0; k < n; ++k) {
        if (!P.admissible(kind[k], T[k])) return -1;
        req[(size_t)k].id = k;
        req[(size_t)k].T = T[k];
        req[(size_t)k].kind = kind[k];
    }
    struct Live {
        int64_t iter, step;
    };
    std::deque<Live> live;
    int64_t nb = 0, ni = 0, step = 0, idle = 0;
    int next = 0;
    int finished = 0;
    auto complete_oldest = [&](int64_t at) {
        iters[live.front().iter * 5 + 1] = (uint64_t)at;
        live.pop_front();
        P.release_oldest();
    };
    while (finished < n || !live.empty()) {
        while (next < n && arrive[next] <= step) P.enqueue(&req[(size_t)next++]);
        while (!live.empty() && step - live.front().step >= lag) complete_oldest(step);
        IterPlan it;
        bool planned = false;
        if (P.has_work()) {
            planned = P.plan(&it);
            if (!planned && !live.empty()) {
                complete_oldest(step);
                planned = P.plan(&it);
            }
        }
        if (planned) {
            if (ni >= cap_iters) return -2;
            uint64_t *row = iters + ni * 5;
            row[0] = (uint64_t)step;
            row[1] = 0;
            row[2] = it.offset;
            row[3] = it.lay.bytes;
            row[4] = P.ring().in_use();
            auto put = [&](const Block &b, int call) {
                int64_t *o = blocks + nb * 9;
                o[0] = ni;
                o[1] = b.req->id;
                o[2] = b.row0;
                o[3] = b.rows;
                o[4] = b.pos;
                o[5] = call;
                o[6] = b.carried;
                o[7] = b.last;
                o[8] = b.fpos;
                ++nb;
                if (b.last) ++finished;
            };
            if (nb + (int64_t)it.fwd.size() + (int64_t)it.adapt.size() > cap_blocks) return -2;
            for (const Block &b : it.fwd) put(b, 0);
            for (const Block &b : it.adapt) put(b, 1);
            live.push_back({ni, step});
            ++ni;
            idle = 0;
        } else if (!live.empty() && next >= n) {
            complete_oldest(step);
        } else if (++idle > 1000000) {
            return -3;
        }
        ++step;
    }
    *n_blocks = nb;
    *n_iters = ni;
    return 0;
}

// The region layout of one iteration (serve_plan.h; frames_f < 0 for
// streamed rows): 15 uint64 offsets
//   a_f e_f s_f a_a e_a gs_a s_a ge_a ga_a tab off_f off_a cont tab_bytes bytes
int lp_plan_layout(int M, int64_t rows_f, int n_f, int64_t rows_a, int n_a, int n_cont, int64_t frames_f,
                   int64_t frames_a, uint64_t *out) {
    if (out == nullptr) return -1;
    const Layout L = layout(M, rows_f, n_f, rows_a, n_a, n_cont, frames_f, frames_a);
    const uint64_t v[15] = {L.a_f, L.e_f, L.s_f, L.a_a, L.e_a, L.gs_a, L.s_a, L.ge_a, L.ga_a,
                            L.tab, L.off_f, L.off_a, L.cont, L.tab_bytes, L.bytes};
    for (int k = 0; k < 15; ++k) out[k] = v[k];
    return 0;
}

uint64_t lp_plan_max_region_bytes(int M, int64_t block_rows, int max_signals, int64_t max_iter_rows) {
    PlanConfig c;
    c.M = M;
    c.block_rows = block_rows;
    c.max_signals = max_signals;
    c.max_iter_rows = max_iter_rows;
    return max_region_bytes(c);
}

}  // extern "C"
