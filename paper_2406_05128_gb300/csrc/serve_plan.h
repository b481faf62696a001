// Continuous-batching planner of the serving loop: host logic only (no CUDA),
// so the same code runs inside the engine and in a CPU-only simulation.
//
// The serving loop runs the time-varying LP filter (Eq. 5 forward; Eq. 11
// and Eq. 12 for requests that also want gradients) for requests that arrive
// at any time.  Work is organised in iterations.  One iteration is at most
// two varlen calls over rows packed back to back in one device region:
//   - a synthesis call (forward only).  A synthesis request advances by a
//     block of at most `block_rows` rows per iteration; a request with rows
//     left continues in the next iteration from the filter state its block
//     ended in (the last M outputs, kept on the device), so a long utterance
//     never holds back the requests that arrive behind it;
//   - an adaptation call (forward + adjoint) over whole requests, since the
//     adjoint runs backwards in time from the end of the signal.
// Continuing blocks come first in every iteration, in the order of the
// previous one; then waiting requests are admitted in arrival order while
// the iteration's call sizes and the device memory budget (a FIFO ring of
// iteration regions) allow.  Admission stops at the first request that does
// not fit (no overtaking), so every request is served in bounded time.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <vector>

namespace tvlp_serve {

enum Kind : int { SYNTH = 0, ADAPT = 1 };

struct PlanConfig {
    int M = 22;                        // filter order of every request
    int64_t block_rows = 96000;        // synthesis rows per request per iteration (even, >= M); 0: whole
    int max_signals = 256;             // signals per call (each of the two calls)
    int64_t max_iter_rows = 4 << 20;   // packed rows per iteration, both calls together
    uint64_t ring_bytes = 0;           // device bytes for iteration regions
    int hop = 0;                       // > 0: synthesis requests carry frames (block_rows a multiple of hop)
};

// Frames of `rows` samples at this hop: ceil(rows / hop) + 1.
inline int64_t frames_of(int64_t rows, int hop) { return (rows + hop - 1) / hop + 1; }

// The planner's view of one request; `user` belongs to the caller.
struct Request {
    int64_t id = 0;
    int64_t T = 0;
    int kind = SYNTH;
    int64_t next_row = 0;  // first row not yet given to an iteration
    bool started = false;
    void *user = nullptr;
};

// One request's rows [row0, row0 + rows) at packed row `pos` of its call.
// Rows are padded to an even count (16-byte aligned coefficient rows for the
// next signal); the pad rows belong to this signal's call slot and carry zero
// inputs.
struct Block {
    Request *req = nullptr;
    int64_t row0 = 0, rows = 0, pos = 0;
    int64_t fpos = 0;      // frames mode: first frame of the block in the call's frame rows
    bool carried = false;  // starts from a carried filter state
    bool last = false;     // the request's final block
};

inline int64_t padded(int64_t rows) { return rows + (rows & 1); }
inline uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Byte offsets of one iteration region: the synthesis call's a (or, in
// frames mode, its frame rows), e, s; the adaptation call's a, e, gs, s, ge,
// ga; then the tables that go to the device in one copy: both calls' row
// offsets, in frames mode the synthesis blocks' first frames, and the
// indexes (into the synthesis call) of the blocks whose request continues.
struct Layout {
    uint64_t a_f = 0, e_f = 0, s_f = 0;
    uint64_t a_a = 0, e_a = 0, gs_a = 0, s_a = 0, ge_a = 0, ga_a = 0;
    uint64_t tab = 0, off_f = 0, off_a = 0, foff = 0, foff_a = 0, cont = 0, tab_bytes = 0;
    uint64_t bytes = 0;
};

// frames_f < 0: streamed coefficient rows; >= 0: frames mode, with frames_f
// frame rows in the synthesis call and frames_a in the adaptation call (whose
// a and ga regions then hold frames: k in, dL/dk out)
inline Layout layout(int M, int64_t rows_f, int n_f, int64_t rows_a, int n_a, int n_cont, int64_t frames_f = -1,
                     int64_t frames_a = 0) {
    Layout L;
    uint64_t p = 0;
    auto take = [&p](uint64_t nbytes) {
        const uint64_t at = p;
        p = align256(p + nbytes);
        return at;
    };
    const uint64_t rf = (uint64_t)rows_f, ra = (uint64_t)rows_a, m = (uint64_t)M;
    if (n_f > 0) {
        L.a_f = take((frames_f < 0 ? rf : (uint64_t)frames_f) * m * 4);
        L.e_f = take(rf * 4);
        L.s_f = take(rf * 4);
    }
    const uint64_t rk = frames_f < 0 ? ra : (uint64_t)frames_a;  // coefficient rows of the adaptation call
    if (n_a > 0) {
        L.a_a = take(rk * m * 4);
        L.e_a = take(ra * 4);
        L.gs_a = take(ra * 4);
        L.s_a = take(ra * 4);
        L.ge_a = take(ra * 4);
        L.ga_a = take(rk * m * 4);
    }
    L.tab = p;
    L.off_f = p;
    L.off_a = L.off_f + (uint64_t)(n_f + 1) * 8;
    L.foff = L.off_a + (uint64_t)(n_a + 1) * 8;
    L.foff_a = L.foff + (frames_f < 0 ? 0 : (uint64_t)n_f * 8);
    L.cont = L.foff_a + (frames_f < 0 ? 0 : (uint64_t)n_a * 8);
    L.tab_bytes = L.cont + (uint64_t)n_cont * 4 - L.tab;
    p = align256(L.cont + (uint64_t)n_cont * 4);
    L.bytes = p;
    return L;
}

// Largest region one iteration can need (every row in the adaptation call,
// the larger per-row footprint): the ring must hold at least this much so
// that continuing blocks always fit once older iterations have completed.
inline uint64_t max_region_bytes(const PlanConfig &c) {
    const Layout a = layout(c.M, c.max_iter_rows, 0, c.max_iter_rows, c.max_signals, 0);
    const Layout f = layout(c.M, c.max_iter_rows, c.max_signals, 0, 0, c.max_signals);
    return std::max(a.bytes, f.bytes) + 2 * align256((uint64_t)(4 * c.max_signals + 2) * 8 + c.max_signals * 4);
}

// FIFO ring of regions: allocated in iteration order, freed oldest first.
class Ring {
  public:
    explicit Ring(uint64_t cap = 0) : cap_(cap) {}
    uint64_t capacity() const { return cap_; }
    uint64_t in_use() const { return used_; }
    uint64_t peak() const { return peak_; }
    size_t live() const { return live_.size(); }

    // Offset where `nbytes` would go now, or false.
    bool where(uint64_t nbytes, uint64_t *off) const {
        nbytes = std::max<uint64_t>(align256(nbytes), 256);
        if (nbytes > cap_) return false;
        if (live_.empty()) {
            *off = 0;
            return true;
        }
        const Region &front = live_.front(), &back = live_.back();
        if (back.off >= front.off) {  // occupied span [front.off, back.end)
            if (back.end + nbytes <= cap_) {
                *off = back.end;
                return true;
            }
            if (nbytes <= front.off) {
                *off = 0;
                return true;
            }
            return false;
        }
        // wrapped: free space is [back.end, front.off)
        if (back.end + nbytes <= front.off) {
            *off = back.end;
            return true;
        }
        return false;
    }
    bool alloc(uint64_t nbytes, uint64_t *off) {
        if (!where(nbytes, off)) return false;
        nbytes = std::max<uint64_t>(align256(nbytes), 256);
        live_.push_back({*off, *off + nbytes});
        used_ += nbytes;
        peak_ = std::max(peak_, used_);
        return true;
    }
    void free_oldest() {
        if (live_.empty()) return;
        used_ -= live_.front().end - live_.front().off;
        live_.pop_front();
    }

  private:
    struct Region {
        uint64_t off, end;
    };
    uint64_t cap_ = 0, used_ = 0, peak_ = 0;
    std::deque<Region> live_;
};

struct IterPlan {
    std::vector<Block> fwd;    // synthesis call: continuing blocks first
    std::vector<Block> adapt;  // adaptation call: whole requests
    std::vector<int> cont;     // indexes into fwd of blocks whose request continues
    int n_carried = 0;         // fwd[0 .. n_carried) start from a carried state
    int64_t rows_f = 0, rows_a = 0;
    int64_t frames_f = 0;  // frames mode: frame rows of the synthesis call
    int64_t frames_a = 0;  // frames mode: frame rows of the adaptation call
    Layout lay;
    uint64_t offset = 0;  // region offset in the ring
};

class Planner {
  public:
    explicit Planner(const PlanConfig &c) : cfg_(c), ring_(c.ring_bytes) {}
    const PlanConfig &config() const { return cfg_; }
    const Ring &ring() const { return ring_; }
    size_t waiting() const { return wait_.size(); }
    size_t continuing() const { return cont_.size(); }
    bool has_work() const { return !wait_.empty() || !cont_.empty(); }

    // Rows of the first block of a request of this kind and length.
    int64_t first_rows(int kind, int64_t T) const {
        if (kind == ADAPT || cfg_.block_rows <= 0) return T;
        return std::min(T, cfg_.block_rows);
    }
    // Whether a request could ever be planned (alone, in an empty ring).
    bool admissible(int kind, int64_t T) const {
        if (T < 0) return false;
        const int64_t r = padded(first_rows(kind, T));
        if (r > cfg_.max_iter_rows) return false;
        const Layout L = kind == ADAPT ? layout(cfg_.M, 0, 0, r, 1, 0) : layout(cfg_.M, r, 1, 0, 0, 1);
        return align256(L.bytes) <= ring_.capacity();
    }

    void enqueue(Request *r) { wait_.push_back(r); }

    // Plan the next iteration into `out`.  Returns false when there is no
    // work, or when the ring cannot hold even the continuing blocks yet (the
    // caller then waits for the oldest iteration to complete).
    bool plan(IterPlan *out) {
        IterPlan &P = *out;
        P = IterPlan();
        const int64_t S = cfg_.block_rows;
        auto block_of = [&](Request *r) {
            Block b;
            b.req = r;
            b.row0 = r->next_row;
            const int64_t left = r->T - r->next_row;
            b.rows = (r->kind == ADAPT || S <= 0) ? left : std::min(left, S);
            b.last = b.row0 + b.rows >= r->T;
            b.carried = r->started;
            return b;
        };
        int n_cont_next = 0;
        const bool frames = cfg_.hop > 0;
        // frame rows a synthesis block needs (frames mode)
        auto nfr = [&](int64_t rows) { return frames ? frames_of(padded(rows), cfg_.hop) : 0; };
        for (Request *r : cont_) {
            Block b = block_of(r);
            b.pos = P.rows_f;
            b.fpos = P.frames_f;
            P.rows_f += padded(b.rows);
            P.frames_f += nfr(b.rows);
            if (!b.last) ++n_cont_next;
            P.fwd.push_back(b);
        }
        P.n_carried = (int)P.fwd.size();
        uint64_t off = 0;
        auto lay_of = [&](int64_t rf, int nf, int64_t ra, int na, int nc, int64_t ff, int64_t fa) {
            return layout(cfg_.M, rf, nf, ra, na, nc, frames ? ff : -1, fa);
        };
        auto fits = [&](int64_t rf, int nf, int64_t ra, int na, int nc, int64_t ff, int64_t fa) {
            if (rf + ra > cfg_.max_iter_rows) return false;
            if (nf > cfg_.max_signals || na > cfg_.max_signals) return false;
            return ring_.where(lay_of(rf, nf, ra, na, nc, ff, fa).bytes, &off);
        };
        if (!P.fwd.empty() && !fits(P.rows_f, (int)P.fwd.size(), 0, 0, n_cont_next, P.frames_f, 0)) {
            P = IterPlan();
            return false;
        }
        size_t admitted = 0;
        for (; admitted < wait_.size(); ++admitted) {
            Request *r = wait_[admitted];
            Block b = block_of(r);
            const int64_t pr = padded(b.rows);
            if (r->kind == ADAPT) {
                const int64_t fa = P.frames_a + nfr(b.rows);
                if (!fits(P.rows_f, (int)P.fwd.size(), P.rows_a + pr, (int)P.adapt.size() + 1, n_cont_next,
                          P.frames_f, fa))
                    break;
                b.pos = P.rows_a;
                b.fpos = P.frames_a;
                P.rows_a += pr;
                P.frames_a = fa;
                P.adapt.push_back(b);
            } else {
                const int nc = n_cont_next + (b.last ? 0 : 1);
                const int64_t ff = P.frames_f + nfr(b.rows);
                if (!fits(P.rows_f + pr, (int)P.fwd.size() + 1, P.rows_a, (int)P.adapt.size(), nc, ff, P.frames_a))
                    break;
                b.pos = P.rows_f;
                b.fpos = P.frames_f;
                P.rows_f += pr;
                P.frames_f = ff;
                n_cont_next = nc;
                P.fwd.push_back(b);
            }
        }
        if (P.fwd.empty() && P.adapt.empty()) return false;
        // the last successful fits() sized exactly this layout, so the
        // allocation succeeds
        P.lay = lay_of(P.rows_f, (int)P.fwd.size(), P.rows_a, (int)P.adapt.size(), n_cont_next, P.frames_f,
                       P.frames_a);
        if (!ring_.alloc(P.lay.bytes, &P.offset)) {
            P = IterPlan();
            return false;
        }
        wait_.erase(wait_.begin(), wait_.begin() + (std::ptrdiff_t)admitted);
        std::vector<Request *> next;
        for (int k = 0; k < (int)P.fwd.size(); ++k) {
            Block &b = P.fwd[k];
            b.req->started = true;
            b.req->next_row = b.row0 + b.rows;
            if (!b.last) {
                P.cont.push_back(k);
                next.push_back(b.req);
            }
        }
        for (Block &b : P.adapt) {
            b.req->started = true;
            b.req->next_row = b.req->T;
        }
        cont_.swap(next);
        return true;
    }

    // The oldest planned iteration has completed: its region is free.
    void release_oldest() { ring_.free_oldest(); }

  private:
    PlanConfig cfg_;
    Ring ring_;
    std::deque<Request *> wait_;
    std::vector<Request *> cont_;
};

}  // namespace tvlp_serve
