"""Pins of the frame-wise overlap-add oracle (the approximation of Eq. 5
that the paper's sample-wise filter replaces, Sec. 3.2; 75 % overlap as in
Sec. 5.2), checked against things other than itself:

* zero coefficients: the four scaled Hann windows over every sample sum to
  one, so s = e and dL/de = dL/ds exactly (up to rounding);
* each frame's filter is scipy.signal.lfilter's time-invariant all-pole
  filter (Eq. 2) from zero state;
* M = 1: an impulse gives the closed form sum_f w(t0 - t_f) (-a_f)^(t - t0)
  over the frames holding both samples;
* the adjoint: finite differences of <g, s> with respect to every
  excitation sample and every frame coefficient, and the dot-product
  identity <gs, S e> = <ge, e> of the linear map e -> s.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2406_05128_gb300 import inputs

HOP = 8  # small frames keep the brute-force checks quick


def _frames(rng, B, T, M, hop, kmax=0.8):
    F = O.framewise_frames(T, hop)
    k = inputs.reflection_frames(rng, B, F, M, kmax)
    return inputs.step_up(k)


def test_zero_coefficients_identity():
    rng = np.random.default_rng(0)
    T, M = 203, 5
    af = np.zeros((2, O.framewise_frames(T, HOP), M))
    e = rng.standard_normal((2, T))
    gs = rng.standard_normal((2, T))
    s, ge, gaf = O.framewise(af, e, gs, hop=HOP)
    assert np.abs(s - e).max() < 1e-13
    assert np.abs(ge - gs).max() < 1e-13


@pytest.mark.parametrize("M", [1, 4, 10])
def test_frames_are_lfilter(M):
    """Every frame is the time-invariant filter 1/A(z) from zero state on the
    windowed excitation (scipy.signal.lfilter), and the frames overlap-add."""
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(M)
    T, hop = 101, 6
    N = 4 * hop
    af = _frames(rng, 1, T, M, hop)
    e = rng.standard_normal((1, T))
    s = O.framewise(af, e, hop=hop)
    F = af.shape[1]
    want = np.zeros(T + 8 * N)
    n = np.arange(N)
    win = 0.5 - 0.5 * np.cos(2 * np.pi * n / N)
    ep = np.concatenate([np.zeros(4 * N), e[0], np.zeros(4 * N)])
    for f in range(F):
        t0 = (f - 3) * hop + 4 * N
        y = signal.lfilter([1.0], np.concatenate([[1.0], af[0, f]]), 0.5 * win * ep[t0:t0 + N])
        want[t0:t0 + N] += y
    assert np.abs(s[0] - want[4 * N:4 * N + T]).max() < 1e-12


def test_m1_impulse_closed_form():
    rng = np.random.default_rng(3)
    T, hop = 60, 5
    N = 4 * hop
    F = O.framewise_frames(T, hop)
    a = rng.uniform(-0.9, 0.9, size=(1, F, 1))
    t0 = 23
    e = np.zeros((1, T))
    e[0, t0] = 1.0
    s = O.framewise(a, e, hop=hop)[0]
    want = np.zeros(T)
    for t in range(T):
        for f in range(F):
            tf = (f - 3) * hop
            if tf <= t0 <= t < tf + N:
                w = 0.25 * (1 - np.cos(2 * np.pi * (t0 - tf) / N))
                want[t] += w * (-a[0, f, 0]) ** (t - t0)
    assert np.abs(s - want).max() < 1e-14


def test_adjoint_finite_differences():
    rng = np.random.default_rng(7)
    T, M, hop = 37, 3, 4
    af = _frames(rng, 1, T, M, hop, kmax=0.7)
    e = rng.standard_normal((1, T))
    g = rng.standard_normal((1, T))
    _, ge, gaf = O.framewise(af, e, g, hop=hop)
    loss = lambda af_, e_: float((g * O.framewise(af_, e_, hop=hop)).sum())
    h = 1e-6
    for t in range(T):
        d = np.zeros_like(e)
        d[0, t] = h
        fd = (loss(af, e + d) - loss(af, e - d)) / (2 * h)
        assert abs(fd - ge[0, t]) < 1e-7 * max(1.0, abs(fd))
    for f in range(af.shape[1]):
        for i in range(M):
            d = np.zeros_like(af)
            d[0, f, i] = h
            fd = (loss(af + d, e) - loss(af - d, e)) / (2 * h)
            assert abs(fd - gaf[0, f, i]) < 1e-6 * max(1.0, abs(fd)), (f, i, fd, gaf[0, f, i])


def test_adjoint_dot_product_identity():
    rng = np.random.default_rng(11)
    T, M, hop = 500, 8, 20
    af = _frames(rng, 2, T, M, hop)
    e = rng.standard_normal((2, T))
    gs = rng.standard_normal((2, T))
    s, ge, _ = O.framewise(af, e, gs, hop=hop)
    lhs = (gs * s).sum(axis=1)
    rhs = (ge * e).sum(axis=1)
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(lhs).max()
