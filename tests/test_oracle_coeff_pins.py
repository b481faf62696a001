"""Pins of the oracle's coefficient preparation (Sec. 4.3): frame-rate
reflection coefficients, linearly interpolated per sample, stepped up to the
direct form; and of its adjoint dL/dk.

- The step-up is the Levinson recursion: with every frame equal, a(t) must be
  the order-M solution of the Yule-Walker equations that
  scipy.linalg.solve_toeplitz returns, and k_m the last coefficient of its
  order-m solution (reflection coefficients in the A(z) = 1 + sum a_i z^-i
  convention).
- Closed forms: M = 1 gives a_1 = k_1; M = 2 gives a_1 = k_1 (1 + k_2),
  a_2 = k_2 at the frame anchors.  Interpolation: a(t) at t = f hop is the
  step-up of frame f; for M = 1, a_1 is linear between anchors.
- Stability (Schur-Cohn): |k| < 1 makes every root of A(z) lie inside the
  unit circle.
- The adjoint against central finite differences of <ga, a(k)> with respect
  to every frame coefficient, and a closed form for M = 1.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O

scipy_linalg = pytest.importorskip("scipy.linalg")


def _frames_const(kvec, T, hop):
    return np.tile(np.asarray(kvec, np.float64)[None], (O.n_frames(T, hop), 1))


@pytest.mark.parametrize("M", [1, 3, 8, 22])
def test_step_up_is_levinson(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal(8192)
    x = np.convolve(x, rng.standard_normal(6), mode="same")  # a coloured spectrum
    r = np.array([x[: len(x) - j] @ x[j:] for j in range(M + 1)]) / len(x)
    k = np.empty(M)
    for m in range(1, M + 1):
        am = scipy_linalg.solve_toeplitz(r[:m], -r[1:m + 1])
        k[m - 1] = am[m - 1]
    want = scipy_linalg.solve_toeplitz(r[:M], -r[1:M + 1])
    T, hop = 10, 4
    a = O.coeffs(_frames_const(k, T, hop), T, hop)
    for t in range(T):
        np.testing.assert_allclose(a[t], want, rtol=1e-9, atol=1e-12)


def test_closed_forms_at_frame_anchors():
    rng = np.random.default_rng(3)
    T, hop = 40, 8
    k1 = rng.uniform(-0.9, 0.9, (O.n_frames(T, hop), 1))
    a1 = O.coeffs(k1, T, hop)
    k2 = rng.uniform(-0.9, 0.9, (O.n_frames(T, hop), 2))
    a2 = O.coeffs(k2, T, hop)
    for f in range(T // hop):
        t = f * hop
        assert a1[t, 0] == k1[f, 0]
        np.testing.assert_allclose(a2[t], [k2[f, 0] * (1 + k2[f, 1]), k2[f, 1]], rtol=1e-15)
    # M = 1: a_1(t) is linear between anchors (second differences vanish)
    for f in range(T // hop):
        seg = a1[f * hop:(f + 1) * hop + 1 if (f + 1) * hop < T else T, 0]
        np.testing.assert_allclose(np.diff(seg, 2), 0.0, atol=1e-15)
        if (f + 1) * hop < T:
            assert abs(a1[(f + 1) * hop, 0] - k1[f + 1, 0]) < 1e-15


def test_midpoint_is_the_step_up_of_the_mean_frame():
    rng = np.random.default_rng(4)
    M, hop, T = 6, 10, 30
    k = rng.uniform(-0.9, 0.9, (O.n_frames(T, hop), M))
    a = O.coeffs(k, T, hop)
    for f in range(T // hop):
        mid = 0.5 * (k[f] + k[f + 1])
        want = O.coeffs(_frames_const(mid, 1, 1), 1, 1)[0]
        np.testing.assert_allclose(a[f * hop + hop // 2], want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("M", [2, 10, 22])
def test_stable_reflection_coefficients_give_minimum_phase(M):
    rng = np.random.default_rng(10 + M)
    for _ in range(20):
        k = rng.uniform(-0.95, 0.95, M)
        a = O.coeffs(_frames_const(k, 1, 1), 1, 1)[0]
        roots = np.roots(np.concatenate([[1.0], a]))
        assert np.max(np.abs(roots)) < 1.0
    # and one |k_m| > 1 puts a root outside
    k = rng.uniform(-0.5, 0.5, M)
    k[M // 2] = 1.5
    a = O.coeffs(_frames_const(k, 1, 1), 1, 1)[0]
    assert np.max(np.abs(np.roots(np.concatenate([[1.0], a])))) > 1.0


@pytest.mark.parametrize("M,T,hop", [(1, 9, 4), (3, 13, 4), (5, 11, 3)])
def test_adjoint_finite_differences(M, T, hop):
    rng = np.random.default_rng(100 + M)
    k = rng.uniform(-0.8, 0.8, (O.n_frames(T, hop), M))
    ga = rng.standard_normal((T, M))
    gk = O.coeffs_adjoint(k, ga, hop)
    h = 1e-6
    fd = np.zeros_like(k)
    for f in range(k.shape[0]):
        for m in range(M):
            kp, km = k.copy(), k.copy()
            kp[f, m] += h
            km[f, m] -= h
            fd[f, m] = (np.sum(ga * O.coeffs(kp, T, hop)) - np.sum(ga * O.coeffs(km, T, hop))) / (2 * h)
    np.testing.assert_allclose(gk, fd, rtol=1e-7, atol=1e-9)


def test_adjoint_closed_form_m1():
    """M = 1, ga = 1: frame f receives sum (1 - w) over its own segment and
    sum w over the previous one; hop 4 gives 2.5 and 1.5."""
    hop, T = 4, 12
    k = np.random.default_rng(5).uniform(-0.5, 0.5, (O.n_frames(T, hop), 1))
    gk = O.coeffs_adjoint(k, np.ones((T, 1)), hop)
    np.testing.assert_allclose(gk[:, 0], [2.5, 4.0, 4.0, 1.5], rtol=1e-15)
