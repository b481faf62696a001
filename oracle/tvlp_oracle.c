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
