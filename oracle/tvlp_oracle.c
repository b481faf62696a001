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
