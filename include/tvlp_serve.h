/*
 * tvlp_serve.h — C ABI of the serving loop of the time-varying LP library.
 *
 * A server runs the filter of tvlp.h (Eq. 5 forward; Eq. 11 adjoint and
 * Eq. 12 coefficient gradient of arXiv 2406.05128) for requests that arrive
 * one at a time from any host thread, with continuous batching on one GPU.
 * The paper trains and evaluates offline and has no serving loop; this is
 * an extension.
 *
 * Requests
 *   kind LP_SERVE_SYNTH   forward only:  s = LP_a(e)           (Eq. 5)
 *   kind LP_SERVE_ADAPT   forward and adjoint: s, ge, ga for a given gs
 *                         (Eq. 5, Eq. 11, Eq. 12)
 * Every request is one signal of T samples with zero initial state, at the
 * server's order M, FP32, with HOST buffers laid out as in tvlp.h:
 *   a [T][M], e [T], gs [T] (inputs);  s [T], ge [T], ga [T][M] (outputs).
 * Buffers should be page-locked (cudaHostAlloc / cudaHostRegister) so that
 * copies overlap with compute.  The caller keeps every buffer of a request
 * alive and unchanged until lp_serve_poll has returned the request's id.
 *
 * Scheduling
 *   A worker thread owned by the server forms iterations.  One iteration is
 *   at most two varlen calls (lp_tv_forward_varlen_f32, and for
 *   adaptation requests lp_tv_backward_varlen_f32 with
 *   LP_BWD_REUSE_FORWARD) over the iteration's rows, packed in one region
 *   of device memory:
 *   - synthesis requests advance by blocks of at most `block_rows` samples;
 *     a request with samples left continues in the next iteration from the
 *     last M outputs of its block (its filter state, which stays on the
 *     device: s(-j) of the next block is s(end-j) of this one);
 *   - adaptation requests run whole (the adjoint runs from the end of the
 *     signal backwards).
 *   Continuing blocks come first; waiting requests are then admitted in
 *   arrival order while the iteration stays within max_signals signals per
 *   call, max_iter_rows rows, and the device memory left in the server's
 *   budget.  Admission stops at the first request that does not fit.
 *   Up to max_inflight iterations are in flight: the host-to-device copies
 *   of one, the kernels of another and the device-to-host copies of a third
 *   run at the same time on three streams.
 * Every call of the server uses the same chunk length, and a signal's
 * results from a varlen call do not depend on the other signals of the call
 * (tvlp.h), and the blocks of a request depend only on its length: so a
 * request's results are bit for bit the same whatever else is in flight.
 *
 * Device memory: lp_serve_create allocates, once, `hbm_budget` bytes at most
 * (workspace, filter states, and a ring of iteration regions); nothing is
 * allocated later.
 *
 * Latency: the time from the request's arrival (the `arrival_ns` given to
 * lp_serve_submit on the lp_serve_now_ns clock, or the submit call itself)
 * to the moment the worker sees the request's last device-to-host copy
 * complete.
 *
 * Return values are LP_OK or the negative codes of tvlp.h.  A failed CUDA
 * call inside the worker puts the server in an error state: every request
 * still in it completes with that status and later submits return it.
 */
#ifndef TVLP_SERVE_H
#define TVLP_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "tvlp.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { LP_SERVE_SYNTH = 0, LP_SERVE_ADAPT = 1 };

typedef struct lp_serve_config {
    int M;                 /* filter order of every request, 1..32            */
    int chunk;             /* scan chunk length of every call; 0: picked once  */
    int64_t block_rows;    /* synthesis samples per request per iteration;
                              rounded up to even, >= M; 0: whole requests      */
    int max_signals;       /* signals per call, >= 1                          */
    int64_t max_iter_rows; /* packed rows per iteration, both calls           */
    int max_inflight;      /* iterations in flight, 1..16                     */
    uint64_t hbm_budget;   /* device bytes the server may hold                */
    int hop;               /* 0: requests carry a [T][M].  > 0: requests
                              carry reflection coefficients per frame
                              k [ceil(T/hop)+1][M] (as in
                              lp_tv_forward_frames_f32) in place of a, the
                              kernels generate a(t), and an adaptation request
                              receives dL/dk [ceil(T/hop)+1][M] in place of
                              ga; block_rows is rounded up to a multiple of
                              hop                                              */
} lp_serve_config;

typedef struct lp_serve_stats {
    int64_t submitted, completed;
    int64_t iterations;       /* iterations issued                              */
    int64_t synth_calls;      /* forward varlen calls                           */
    int64_t adapt_calls;      /* forward + adjoint varlen call pairs            */
    int64_t kernel_launches;  /* kernels the worker launched                    */
    int64_t blocks;           /* synthesis blocks                               */
    int64_t carried_blocks;   /* ... of them starting from a carried state      */
    int64_t rows;             /* samples processed (both calls, no padding)     */
    int64_t max_signals_iter; /* most signals in one iteration                  */
    int64_t max_waiting;      /* longest admission queue seen                   */
    int64_t overlapped;       /* iterations issued while another was in flight  */
    uint64_t device_bytes;    /* device memory held by the server               */
    uint64_t ring_bytes;      /* ... of it for iteration regions                */
    uint64_t ring_peak;       /* most ring bytes in use at once                 */
    int chunk;                /* chunk length every call uses                   */
    int error;                /* LP_OK or the error that stopped the server     */
} lp_serve_stats;

/* Defaults: M = 22, chunk picked, block_rows = 96000, max_signals = 256,
 * max_iter_rows = 4194304, max_inflight = 4, hbm_budget = 20 GiB, hop = 0. */
void lp_serve_default_config(lp_serve_config *cfg);

/* Create a server on the calling thread's current device.  Validates cfg
 * (LP_EINVAL), checks that the budget holds the workspace, the filter
 * states and at least one largest iteration region (LP_ETOOBIG), then
 * allocates device memory (LP_ECUDA if that fails) and starts the worker. */
int lp_serve_create(const lp_serve_config *cfg, void **server);

/* Finish every submitted request, stop the worker and free everything. */
int lp_serve_destroy(void *server);

/* Queue one request (never blocks on the GPU).  kind LP_SERVE_SYNTH needs
 * a, e, s (gs, ge, ga ignored); LP_SERVE_ADAPT needs all six.  T >= 0.
 * arrival_ns <= 0 stamps the arrival now.  With hop > 0, `a` points to the
 * request's frames and `ga` receives dL/dk per frame.  Returns LP_EINVAL
 * for a bad argument, LP_ETOOBIG for a request no iteration can hold. */
int lp_serve_submit(void *server, int64_t id, int kind, int64_t T,
                    const float *a, const float *e, const float *gs,
                    float *s, float *ge, float *ga, int64_t arrival_ns);

/* Completed requests since the last call, at most `max`: ids[k],
 * latency_ns[k] and status[k] (LP_OK or the server's error).  Returns how
 * many were written; never blocks. */
int lp_serve_poll(void *server, int64_t *ids, int64_t *latency_ns,
                  int *status, int max);

/* Wait until every submitted request has completed, at most timeout_ms
 * milliseconds (< 0: no limit).  LP_OK, LP_ETIMEOUT or the server error. */
int lp_serve_drain(void *server, int64_t timeout_ms);

/* Counters; with `reset` non-zero, the counters that describe a period
 * (iterations, calls, blocks, rows, maxima, ring peak) restart at zero. */
int lp_serve_stats_get(void *server, lp_serve_stats *st, int reset);

/* The server's clock (monotonic, nanoseconds). */
int64_t lp_serve_now_ns(void);

#ifdef __cplusplus
}
#endif

#endif /* TVLP_SERVE_H */
