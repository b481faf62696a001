/*
 * Sequential FP64 oracle for the differentiable sample-wise time-varying
 * linear-prediction (TV-LP) filter of Yu & Fazekas, "Differentiable
 * Time-Varying Linear Prediction in the Context of End-to-End
 * Analysis-by-Synthesis" (Interspeech 2024, arXiv 2406.05128).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the CUDA library computes.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline / reference legs may load it; the
 * product path never calls it and shares no code with it.
 *
 * Every routine is written in double precision, one signal at a time, in
 * the order the paper states the recursions.  No blocking, no reordering.
 *
 * Layouts (row-major, one signal):
 *   a  [T][M]  a[t*M + (i-1)] = a~_i(t), the i-th LP coefficient at sample t
 *   e  [T]     excitation e(t)
 *   s  [T]     output s(t)
 *   zi [M]     initial state, zi[j-1] = s(-j); NULL means zero (Sec. 2.2)
 *
 * Sample count: the paper indexes samples 0..T (T+1 samples, Sec. 2.2);
 * here a signal has T samples indexed 0..T-1.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

/* s(t - i) for the forward recursion, reading the initial state for t-i<0. */
static double past_output(const double *s, const double *zi, int64_t t, int i)
{
    int64_t k = t - i;
    if (k >= 0)
        return s[k];
    /* k = -j with j = i - t >= 1 */
    return zi ? zi[(i - t) - 1] : 0.0;
}

/*
 * Eq. 5 (Sec. 3.2): s(t) = e(t) - sum_{i=1..M} a~_i(t) s(t-i).
 * With zi == NULL this is the zero-initial-condition filter of Sec. 2.2.
 */
void tvlp_oracle_forward(int64_t T, int M, const double *a, const double *e,
                         const double *zi, double *s)
{
    for (int64_t t = 0; t < T; ++t) {
        double acc = e[t];
        for (int i = 1; i <= M; ++i)
            acc -= a[t * M + (i - 1)] * past_output(s, zi, t, i);
        s[t] = acc;
    }
}

/*
 * Eq. 11 (Sec. 3.2.1): dL/de is the same LP filter run backwards in time
 * (t = T-1 down to 0) on dL/ds, with the lag-shifted coefficients
 * a^_i(t) = a~_i(t+i) (the shift stated just after Eq. 10):
 *     ge(t) = gs(t) - sum_{i=1..M} a^_i(t) ge(t+i),   ge(t) = 0 for t >= T.
 *
 * Eq. 12 (Sec. 3.2.2): dL/da~_i(t) = -dL/de(t) * s(t-i), where s(t-i) for
 * t-i < 0 is the initial state (zero when zi == NULL).
 *
 * Initial-state gradient (an extension; the paper assumes zero initial
 * conditions): s(-j) enters the output at sample t through the term
 * -a~_{t+j}(t) s(-j) of Eq. 5 whenever 1 <= t+j <= M, so by the same chain
 * rule as Eq. 12, dL/ds(-j) = -sum_{t=0}^{M-j} ge(t) a~_{t+j}(t).
 *
 * ga [T][M] and gzi [M] may be NULL.
 */
void tvlp_oracle_backward(int64_t T, int M, const double *a, const double *s,
                          const double *zi, const double *gs, double *ge,
                          double *ga, double *gzi)
{
    for (int64_t t = T - 1; t >= 0; --t) {
        double acc = gs[t];
        for (int i = 1; i <= M; ++i) {
            if (t + i < T) {
                double a_hat = a[(t + i) * M + (i - 1)]; /* a^_i(t) = a~_i(t+i) */
                acc -= a_hat * ge[t + i];
            }
        }
        ge[t] = acc;
    }
    if (ga) {
        for (int64_t t = 0; t < T; ++t)
            for (int i = 1; i <= M; ++i)
                ga[t * M + (i - 1)] = -ge[t] * past_output(s, zi, t, i);
    }
    if (gzi) {
        for (int j = 1; j <= M; ++j) {
            double acc = 0.0;
            for (int64_t t = 0; t <= (int64_t)(M - j) && t < T; ++t)
                acc -= ge[t] * a[t * M + (t + j - 1)];
            gzi[j - 1] = acc;
        }
    }
}

/* Batched forms: B independent signals, arrays stacked along a leading axis. */
void tvlp_oracle_forward_batch(int64_t B, int64_t T, int M, const double *a,
                               const double *e, const double *zi, double *s)
{
    for (int64_t b = 0; b < B; ++b)
        tvlp_oracle_forward(T, M, a + b * T * M, e + b * T,
                            zi ? zi + b * M : NULL, s + b * T);
}

void tvlp_oracle_backward_batch(int64_t B, int64_t T, int M, const double *a,
                                const double *s, const double *zi,
                                const double *gs, double *ge, double *ga,
                                double *gzi)
{
    for (int64_t b = 0; b < B; ++b)
        tvlp_oracle_backward(T, M, a + b * T * M, s + b * T,
                             zi ? zi + b * M : NULL, gs + b * T, ge + b * T,
                             ga ? ga + b * T * M : NULL,
                             gzi ? gzi + b * M : NULL);
}

/*
 * Sec. 4.3: per-sample coefficients from frame-rate reflection coefficients.
 *   k  [F][M]  k[f*M + (m-1)] = k_m of frame f; frame f sits at sample f*hop
 *              (F = ceil(T/hop) + 1 frames, so the last segment has an end)
 * Linear interpolation between the two frames around t:
 *   f = floor(t / hop), w = (t - f*hop) / hop,  k_m(t) = (1 - w) k_m[f] + w k_m[f+1]
 * then the step-up recursion to the direct form of A(z) = 1 + sum a_i z^-i:
 *   a^(m)_i = a^(m-1)_i + k_m a^(m-1)_{m-i}  (i = 1..m-1),   a^(m)_m = k_m,
 * and a(t) = a^(M).  Orders up to TVLP_ORACLE_MAX_M.
 */
#define TVLP_ORACLE_MAX_M 64

static double interp_k(const double *k, int M, int hop, int64_t t, int m)
{
    int64_t f = t / hop;
    double w = (double)(t - f * hop) / (double)hop;
    return (1.0 - w) * k[f * M + (m - 1)] + w * k[(f + 1) * M + (m - 1)];
}

/* A[m][i] = a^(m)_i for m = 0..M, i = 1..m (row m holds the order-m filter). */
static void step_up(int M, const double *km, double A[][TVLP_ORACLE_MAX_M + 1])
{
    for (int m = 1; m <= M; ++m) {
        for (int i = 1; i < m; ++i)
            A[m][i] = A[m - 1][i] + km[m] * A[m - 1][m - i];
        A[m][m] = km[m];
    }
}

void tvlp_oracle_coeffs(int64_t T, int M, int hop, const double *k, double *a)
{
    double (*A)[TVLP_ORACLE_MAX_M + 1] = malloc(sizeof(double[TVLP_ORACLE_MAX_M + 1][TVLP_ORACLE_MAX_M + 1]));
    double km[TVLP_ORACLE_MAX_M + 1] = {0.0};
    for (int64_t t = 0; t < T; ++t) {
        for (int m = 1; m <= M; ++m)
            km[m] = interp_k(k, M, hop, t, m);
        step_up(M, km, A);
        for (int i = 1; i <= M; ++i)
            a[t * M + (i - 1)] = A[M][i];
    }
    free(A);
}

/*
 * dL/dk from dL/da (ga [T][M]) for the coefficients of tvlp_oracle_coeffs:
 * the chain rule in forward mode.  For every sample the derivatives
 * D[m][i][j] = d a^(m)_i / d k_j(t) follow the step-up term by term,
 *   D[m][i][j] = D[m-1][i][j] + k_m D[m-1][m-i][j] + [j == m] a^(m-1)_{m-i}
 *   D[m][m][j] = [j == m],
 * then dL/dk_j(t) = sum_i ga_i(t) D[M][i][j], and the interpolation sends
 * (1 - w) of it to frame f and w of it to frame f+1.  gk [F][M] is
 * overwritten (F = ceil(T/hop) + 1).
 */
void tvlp_oracle_coeffs_adjoint(int64_t T, int M, int hop, const double *k,
                                const double *ga, double *gk)
{
    double (*A)[TVLP_ORACLE_MAX_M + 1] = malloc(sizeof(double[TVLP_ORACLE_MAX_M + 1][TVLP_ORACLE_MAX_M + 1]));
    double (*D)[TVLP_ORACLE_MAX_M + 1][TVLP_ORACLE_MAX_M + 1] =
        malloc(sizeof(double[TVLP_ORACLE_MAX_M + 1][TVLP_ORACLE_MAX_M + 1][TVLP_ORACLE_MAX_M + 1]));
    double km[TVLP_ORACLE_MAX_M + 1] = {0.0};
    int64_t F = (T + hop - 1) / hop + 1;
    for (int64_t x = 0; x < F * M; ++x)
        gk[x] = 0.0;
    for (int64_t t = 0; t < T; ++t) {
        for (int m = 1; m <= M; ++m)
            km[m] = interp_k(k, M, hop, t, m);
        step_up(M, km, A);
        for (int m = 1; m <= M; ++m) {
            for (int j = 1; j <= M; ++j) {
                for (int i = 1; i < m; ++i) {
                    double d = D[m - 1][i][j] + km[m] * D[m - 1][m - i][j];
                    if (j == m)
                        d += A[m - 1][m - i];
                    D[m][i][j] = d;
                }
                D[m][m][j] = (j == m) ? 1.0 : 0.0;
            }
        }
        int64_t f = t / hop;
        double w = (double)(t - f * hop) / (double)hop;
        for (int j = 1; j <= M; ++j) {
            double g = 0.0;
            for (int i = 1; i <= M; ++i)
                g += ga[t * M + (i - 1)] * D[M][i][j];
            gk[f * M + (j - 1)] += (1.0 - w) * g;
            gk[(f + 1) * M + (j - 1)] += w * g;
        }
    }
    free(D);
    free(A);
}

/* Batched forms of the coefficient routines: k [B][F][M], a / ga [B][T][M]. */
void tvlp_oracle_coeffs_batch(int64_t B, int64_t T, int M, int hop,
                              const double *k, double *a)
{
    int64_t F = (T + hop - 1) / hop + 1;
    for (int64_t b = 0; b < B; ++b)
        tvlp_oracle_coeffs(T, M, hop, k + b * F * M, a + b * T * M);
}

void tvlp_oracle_coeffs_adjoint_batch(int64_t B, int64_t T, int M, int hop,
                                      const double *k, const double *ga,
                                      double *gk)
{
    int64_t F = (T + hop - 1) / hop + 1;
    for (int64_t b = 0; b < B; ++b)
        tvlp_oracle_coeffs_adjoint(T, M, hop, k + b * F * M, ga + b * T * M,
                                   gk + b * F * M);
}

/*
 * Frame-wise approximation of Eq. 5 (Sec. 3.2, the method of the earlier
 * GOLF work that the sample-wise filter replaces; Sec. 5.2 states the 75 %
 * overlap, Sec. 4.3 lists the frame-wise decoder GOLF-ff).
 * The signal is cut into frames of N = 4*hop samples, one every hop
 * samples; frame f covers samples t_f .. t_f + N - 1 with t_f = (f - 3)*hop,
 * so with F = ceil(T/hop) + 3 frames every sample lies in exactly four.
 * Each frame:
 *   u_f(n) = w(n) e(t_f + n)                  (e = 0 outside 0..T-1)
 *   y_f(n) = u_f(n) - sum_{i=1..M} af_i y_f(n-i),  y_f(n < 0) = 0
 * i.e. the time-invariant filter of Eq. 2 with the frame's coefficients
 * af [F][M], run from zero state over the frame; the outputs overlap-add:
 *   s(t) = sum_f y_f(t - t_f)   over the frames with 0 <= t - t_f < N.
 * w(n) = (1 - cos(2 pi n / N)) / 4, a periodic Hann window scaled so that
 * the four windows over any sample sum to one.  (The paper states the
 * per-frame filtering and the overlap; frame length, window and where it
 * is applied are this build's reading.)
 * y [F][N] may be NULL; it receives the frame outputs.
 */
static double ff_window(int64_t n, int64_t N)
{
    return 0.25 * (1.0 - cos(2.0 * 3.14159265358979323846 * (double)n / (double)N));
}

int64_t tvlp_oracle_framewise_frames(int64_t T, int hop)
{
    return (T + hop - 1) / hop + 3;
}

void tvlp_oracle_framewise_forward(int64_t T, int M, int hop, const double *af,
                                   const double *e, double *s, double *y)
{
    const int64_t N = 4 * (int64_t)hop;
    const int64_t F = tvlp_oracle_framewise_frames(T, hop);
    double *yf = malloc(sizeof(double) * (size_t)N);
    for (int64_t t = 0; t < T; ++t)
        s[t] = 0.0;
    for (int64_t f = 0; f < F; ++f) {
        const int64_t t0 = (f - 3) * hop;
        for (int64_t n = 0; n < N; ++n) {
            const int64_t t = t0 + n;
            double acc = (t >= 0 && t < T) ? ff_window(n, N) * e[t] : 0.0;
            for (int i = 1; i <= M; ++i)
                if (n - i >= 0)
                    acc -= af[f * M + (i - 1)] * yf[n - i];
            yf[n] = acc;
            if (t >= 0 && t < T)
                s[t] += acc;
            if (y)
                y[f * N + n] = acc;
        }
    }
    free(yf);
}

/*
 * Its adjoint for dL/ds = gs: the overlap-add hands every frame
 * g_f(n) = gs(t_f + n); Eq. 11 with the frame's constant coefficients runs
 * backwards over the frame from a zero state past its end,
 *   gu_f(n) = g_f(n) - sum_{i=1..M} af_i gu_f(n+i),  gu_f(n >= N) = 0,
 * the window and the framing send it back to the excitation,
 *   ge(t) = sum_f w(t - t_f) gu_f(t - t_f),
 * and Eq. 12 summed over the frame (Eq. 3) gives the frame's coefficients
 *   gaf_i = -sum_n gu_f(n) y_f(n - i),  y_f(n < 0) = 0.
 * y [F][N] are the forward's frame outputs.
 */
void tvlp_oracle_framewise_backward(int64_t T, int M, int hop, const double *af,
                                    const double *y, const double *gs,
                                    double *ge, double *gaf)
{
    const int64_t N = 4 * (int64_t)hop;
    const int64_t F = tvlp_oracle_framewise_frames(T, hop);
    double *gu = malloc(sizeof(double) * (size_t)N);
    for (int64_t t = 0; t < T; ++t)
        ge[t] = 0.0;
    for (int64_t f = 0; f < F; ++f) {
        const int64_t t0 = (f - 3) * hop;
        for (int64_t n = N - 1; n >= 0; --n) {
            const int64_t t = t0 + n;
            double acc = (t >= 0 && t < T) ? gs[t] : 0.0;
            for (int i = 1; i <= M; ++i)
                if (n + i < N)
                    acc -= af[f * M + (i - 1)] * gu[n + i];
            gu[n] = acc;
            if (t >= 0 && t < T)
                ge[t] += ff_window(n, N) * acc;
        }
        for (int i = 1; i <= M; ++i) {
            double g = 0.0;
            for (int64_t n = i; n < N; ++n)
                g -= gu[n] * y[f * N + (n - i)];
            gaf[f * M + (i - 1)] = g;
        }
    }
    free(gu);
}

/* Batched: af / gaf [B][F][M], e / s / gs / ge [B][T], y [B][F][N]. */
void tvlp_oracle_framewise_batch(int64_t B, int64_t T, int M, int hop,
                                 const double *af, const double *e,
                                 const double *gs, double *s, double *ge,
                                 double *gaf)
{
    const int64_t N = 4 * (int64_t)hop;
    const int64_t F = tvlp_oracle_framewise_frames(T, hop);
    double *y = malloc(sizeof(double) * (size_t)(F * N));
    for (int64_t b = 0; b < B; ++b) {
        tvlp_oracle_framewise_forward(T, M, hop, af + b * F * M, e + b * T,
                                      s + b * T, y);
        if (gs)
            tvlp_oracle_framewise_backward(T, M, hop, af + b * F * M, y,
                                           gs + b * T, ge + b * T,
                                           gaf + b * F * M);
    }
    free(y);
}
