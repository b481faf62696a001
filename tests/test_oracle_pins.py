"""Pins for the FP64 oracle: results fixed by the paper and by mathematics,
not by the oracle itself.

Each test states the passage of Yu & Fazekas (arXiv 2406.05128) or the
mathematical fact it checks.  Together they make a plausible slip in the
oracle (a dropped term, a wrong sign, an off-by-one lag, a transposed
operand, mishandled initial state) fail at least one test;
test_oracle_mutants.py plants such slips and confirms it.
"""
from __future__ import annotations

import itertools
import json
import os

import numpy as np
import pytest
from scipy.signal import lfilter, lfiltic

import oracle as O
from paper_2406_05128_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_a(rng, T, M, scale=0.5):
    return rng.uniform(-scale, scale, size=(T, M))


def _stable_ti(rng, M, rmax=0.95):
    """Direct-form coefficients of a random stable all-pole filter with
    distinct poles (conjugate pairs plus, for odd M, one real pole)."""
    poles = []
    for _ in range(M // 2):
        r = rng.uniform(0.3, rmax)
        th = rng.uniform(0.2, 2.9)
        poles += [r * np.exp(1j * th), r * np.exp(-1j * th)]
    if M % 2:
        poles.append(rng.uniform(-rmax, rmax))
    poly = np.real(np.poly(poles))  # [1, a_1, ..., a_M]
    return poly[1:], np.array(poles)


def _ti(a_vec, T):
    return np.tile(np.asarray(a_vec, np.float64)[None, :], (T, 1))


def _adjoint_runner(fn):
    return fn


# ---------------------------------------------------------------------------
# Hand-worked example (tests/golden/worked_m2_t5.json): exact dyadic values.
# ---------------------------------------------------------------------------
def test_golden_worked_example_exact():
    g = json.load(open(os.path.join(GOLDEN, "worked_m2_t5.json")))
    a = np.array(g["a_rows_t_then_i"])
    e, zi, gs = (np.array(g[k]) for k in ("e", "zi", "gs"))
    s = O.forward(a, e, zi)
    assert np.array_equal(s, np.array(g["s"]))
    ge, ga, gzi = O.backward(a, s, gs, zi)
    assert np.array_equal(ge, np.array(g["ge"]))
    assert np.array_equal(ga, np.array(g["ga"]))
    assert np.array_equal(gzi, np.array(g["gzi"]))


# ---------------------------------------------------------------------------
# Closed forms (Eq. 2 / Eq. 5 with constant or first-order coefficients).
# ---------------------------------------------------------------------------
def test_m1_time_varying_product_form():
    """M=1: s(t) = prod_{tau=1..t} (-a_1(tau)) for e = delta(t); the adjoint
    with gs = delta(t-(T-1)) is ge(t) = prod_{tau=t+1..T-1} (-a_1(tau))."""
    rng = np.random.default_rng(0)
    T = 40
    a = rng.uniform(-1.2, 1.2, size=(T, 1))
    e = np.zeros(T); e[0] = 1.0
    s = O.forward(a, e)
    want = np.array([np.prod(-a[1:t + 1, 0]) for t in range(T)])
    np.testing.assert_allclose(s, want, rtol=1e-13, atol=0)
    gs = np.zeros(T); gs[-1] = 1.0
    ge, _, _ = O.backward(a, s, gs)
    want_ge = np.array([np.prod(-a[t + 1:, 0]) for t in range(T)])
    np.testing.assert_allclose(ge, want_ge, rtol=1e-13, atol=0)


def test_m2_resonator_closed_form():
    """Poles r e^{+-j theta}: a_1 = -2 r cos(theta), a_2 = r^2 and the impulse
    response is r^n sin((n+1) theta) / sin(theta)."""
    r, th, T = 0.97, 0.37, 300
    a = _ti([-2 * r * np.cos(th), r * r], T)
    e = np.zeros(T); e[0] = 1.0
    n = np.arange(T)
    h = r ** n * np.sin((n + 1) * th) / np.sin(th)
    np.testing.assert_allclose(O.forward(a, e), h, rtol=0, atol=1e-12)


@pytest.mark.parametrize("M", [3, 6, 10])
def test_partial_fraction_impulse_response(M):
    """h(n) = sum_k p_k^{n+M-1} / prod_{j!=k} (p_k - p_j) over the poles of
    1/A(z).  For a time-invariant filter the adjoint of Eq. 11 run on
    gs = delta(t-(T-1)) returns the time-reversed impulse response."""
    rng = np.random.default_rng(M)
    a_vec, poles = _stable_ti(rng, M)
    T = 200
    n = np.arange(T)
    h = np.zeros(T, complex)
    for k, p in enumerate(poles):
        den = np.prod([p - q for j, q in enumerate(poles) if j != k])
        h += p ** (n + M - 1) / den
    assert np.max(np.abs(h.imag)) < 1e-9
    a = _ti(a_vec, T)
    e = np.zeros(T); e[0] = 1.0
    s = O.forward(a, e)
    np.testing.assert_allclose(s, h.real, rtol=0, atol=1e-9)
    gs = np.zeros(T); gs[-1] = 1.0
    ge, _, _ = O.backward(a, s, gs)
    np.testing.assert_allclose(ge[::-1], h.real, rtol=0, atol=1e-9)


@pytest.mark.parametrize("M", [1, 4, 12])
def test_time_invariant_matches_lfilter_with_initial_state(M):
    """Constant coefficients reduce Eq. 5 to scipy.signal.lfilter with
    denominator [1, a_1..a_M]; the initial state s(-1..-M) goes through
    scipy.signal.lfiltic."""
    rng = np.random.default_rng(10 + M)
    a_vec, _ = _stable_ti(rng, M, rmax=0.9)
    T = 500
    e = rng.standard_normal(T)
    zi = rng.standard_normal(M)
    den = np.concatenate([[1.0], a_vec])
    want = lfilter([1.0], den, e, zi=lfiltic([1.0], den, y=zi))[0]
    np.testing.assert_allclose(O.forward(_ti(a_vec, T), e, zi), want, rtol=1e-10, atol=1e-10)


# ---------------------------------------------------------------------------
# Brute force: Eq. 5 is the banded unit-lower-triangular system (I + A) s = r
# and Eq. 11 is its transpose (I + A)^T ge = gs.
# ---------------------------------------------------------------------------
def _dense_system(a, e, zi):
    T, M = a.shape
    L = np.eye(T)
    r = np.array(e, np.float64).copy()
    for t in range(T):
        for i in range(1, M + 1):
            if t - i >= 0:
                L[t, t - i] = a[t, i - 1]
            elif zi is not None:
                r[t] -= a[t, i - 1] * zi[i - t - 1]
    return L, r


@pytest.mark.parametrize("T,M", [(1, 1), (5, 3), (3, 7), (33, 4), (64, 9), (20, 20)])
def test_dense_solve_forward_and_adjoint(T, M):
    rng = np.random.default_rng(T * 100 + M)
    a = _rand_a(rng, T, M)
    e, gs = rng.standard_normal(T), rng.standard_normal(T)
    zi = rng.standard_normal(M)
    L, r = _dense_system(a, e, zi)
    s = O.forward(a, e, zi)
    np.testing.assert_allclose(s, np.linalg.solve(L, r), rtol=1e-10, atol=1e-11)
    ge, _, _ = O.backward(a, s, gs, zi)
    np.testing.assert_allclose(ge, np.linalg.solve(L.T, gs), rtol=1e-10, atol=1e-11)


# ---------------------------------------------------------------------------
# Finite differences of J = <g, s> (FP64, central differences).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T,M", [(12, 3), (6, 5), (9, 1)])
def test_finite_differences(T, M):
    rng = np.random.default_rng(7 * T + M)
    a = _rand_a(rng, T, M, 0.6)
    e, g = rng.standard_normal(T), rng.standard_normal(T)
    zi = rng.standard_normal(M)
    J = lambda a_, e_, zi_: float(np.dot(g, O.forward(a_, e_, zi_)))
    s = O.forward(a, e, zi)
    ge, ga, gzi = O.backward(a, s, g, zi)
    h = 1e-6
    fd_a = np.zeros_like(a)
    for t in range(T):
        for i in range(M):
            ap, am = a.copy(), a.copy()
            ap[t, i] += h; am[t, i] -= h
            fd_a[t, i] = (J(ap, e, zi) - J(am, e, zi)) / (2 * h)
    fd_e = np.zeros(T)
    for t in range(T):
        ep, em = e.copy(), e.copy()
        ep[t] += h; em[t] -= h
        fd_e[t] = (J(a, ep, zi) - J(a, em, zi)) / (2 * h)
    fd_z = np.zeros(M)
    for j in range(M):
        zp, zm = zi.copy(), zi.copy()
        zp[j] += h; zm[j] -= h
        fd_z[j] = (J(a, e, zp) - J(a, e, zm)) / (2 * h)
    np.testing.assert_allclose(ga, fd_a, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(ge, fd_e, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(gzi, fd_z, rtol=1e-6, atol=1e-8)


# ---------------------------------------------------------------------------
# The paper's IIR expansion, Eqs. 6-10, enumerated on tiny sizes.
# ---------------------------------------------------------------------------
def _compositions(d, M, memo={}):
    """G_d of Eq. 8: ordered tuples of parts in 1..M summing to d."""
    key = (d, M)
    if key not in memo:
        if d == 0:
            memo[key] = [()]
        else:
            memo[key] = [(i,) + q for i in range(1, min(d, M) + 1)
                         for q in _compositions(d - i, M)]
    return memo[key]


def _b_eq7(a, d, t):
    """Eq. 7: b_d(t) = sum_{q in G_d} (-1)^|q| prod_j a~_{q_j}(t - sum_{k<=j} Q(q)_k),
    Q(q) = [0; q], so the j-th factor is evaluated at t - (q_1 + ... + q_{j-1})."""
    M = a.shape[1]
    total = 0.0
    for q in _compositions(d, M):
        prod, shift = 1.0, 0
        for qj in q:
            prod *= a[t - shift, qj - 1]
            shift += qj
        total += (-1) ** len(q) * prod
    return total


def _b_eq10(a, d, t):
    """Eq. 10, last line: b_d(t+d) from the lag-shifted a^_i(t) = a~_i(t+i),
    the j-th factor evaluated at t + (q_1 + ... + q_{j-1})."""
    M = a.shape[1]
    total = 0.0
    for q in _compositions(d, M):
        prod, shift = 1.0, 0
        for qj in q:
            prod *= a[t + shift + qj, qj - 1]  # a^_{qj}(t + shift)
            shift += qj
        total += (-1) ** len(q) * prod
    return total


@pytest.mark.parametrize("T,M", [(10, 1), (10, 2), (9, 3)])
def test_iir_expansion_eqs_6_to_10(T, M):
    rng = np.random.default_rng(T + 31 * M)
    a = _rand_a(rng, T, M, 0.9)
    e, gs = rng.standard_normal(T), rng.standard_normal(T)
    # Eq. 6: s(t) = e(t) + sum_{d=1..t} b_d(t) e(t-d)
    s_iir = np.array([e[t] + sum(_b_eq7(a, d, t) * e[t - d] for d in range(1, t + 1))
                      for t in range(T)])
    s = O.forward(a, e)
    np.testing.assert_allclose(s, s_iir, rtol=1e-12, atol=1e-12)
    # Eq. 10: the two expressions of b_d(t+d) agree
    for t in range(T):
        for d in range(1, T - t):
            assert abs(_b_eq7(a, d, t + d) - _b_eq10(a, d, t)) < 1e-12
    # Eq. 9: ge(t) = gs(t) + sum_{d=1..T-1-t} b_d(t+d) gs(t+d)
    ge_iir = np.array([gs[t] + sum(_b_eq7(a, d, t + d) * gs[t + d] for d in range(1, T - t))
                       for t in range(T)])
    ge, _, _ = O.backward(a, s, gs)
    np.testing.assert_allclose(ge, ge_iir, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Eqs. 2-3 (GOLF, time-invariant): the two-filter gradient must equal the
# one-filter gradient of Eq. 12 summed over time (Sec. 3.2.2, last paragraph).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("M", [2, 5])
def test_golf_time_invariant_gradients(M):
    rng = np.random.default_rng(50 + M)
    a_vec, _ = _stable_ti(rng, M, rmax=0.9)
    T = 300
    den = np.concatenate([[1.0], a_vec])
    e, g = rng.standard_normal(T), rng.standard_normal(T)
    s = lfilter([1.0], den, e)
    # Eq. 3, first line: dL/da_i = sum_t g(t) LP_a(-s(t-i))
    golf = np.zeros(M)
    for i in range(1, M + 1):
        u = np.concatenate([np.zeros(i), -s[:T - i]])
        golf[i - 1] = np.dot(g, lfilter([1.0], den, u))
    # Eq. 3, second line: dL/de = LP_a run on reversed dL/ds
    golf_ge = lfilter([1.0], den, g[::-1])[::-1]
    a = _ti(a_vec, T)
    ge, ga, _ = O.backward(a, O.forward(a, e), g)
    np.testing.assert_allclose(ge, golf_ge, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ga.sum(axis=0), golf, rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------------------
# Invariants.
# ---------------------------------------------------------------------------
def test_zero_coefficients_are_identity():
    rng = np.random.default_rng(3)
    T, M = 50, 6
    a = np.zeros((T, M))
    e, gs, zi = rng.standard_normal(T), rng.standard_normal(T), rng.standard_normal(M)
    s = O.forward(a, e, zi)
    assert np.array_equal(s, e)
    ge, ga, gzi = O.backward(a, s, gs, zi)
    assert np.array_equal(ge, gs)
    assert np.array_equal(gzi, np.zeros(M))


def test_causality_and_linearity():
    rng = np.random.default_rng(4)
    T, M, t0 = 80, 5, 37
    a = _rand_a(rng, T, M)
    e, zi = rng.standard_normal(T), rng.standard_normal(M)
    s = O.forward(a, e, zi)
    e2 = e.copy(); e2[t0] += 1.0
    s2 = O.forward(a, e2, zi)
    assert np.array_equal(s[:t0], s2[:t0]) and s[t0] != s2[t0]
    e3, zi3 = rng.standard_normal(T), rng.standard_normal(M)
    lhs = O.forward(a, 2.0 * e - 3.0 * e3, 2.0 * zi - 3.0 * zi3)
    rhs = 2.0 * s - 3.0 * O.forward(a, e3, zi3)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_adjoint_dot_product_identity():
    """<g, J de> == <J^T g, de> where J is the map e -> s (zero state)."""
    rng = np.random.default_rng(5)
    T, M = 400, 8
    a = inputs.coefficients(rng, 1, T, M, 0.9, 0.9)[0]
    de, g = rng.standard_normal(T), rng.standard_normal(T)
    lhs = np.dot(g, O.forward(a, de))
    ge, _, _ = O.backward(a, O.forward(a, de), g)
    assert abs(lhs - np.dot(ge, de)) <= 1e-10 * max(1.0, abs(lhs))


def test_slicing_with_carried_state():
    """Running [0,t1) then [t1,T) from the carried state s(t1-1..t1-M)
    reproduces the whole run; the adjoint composes the same way with the
    carried pending gradient (the initial-state gradient of the tail)."""
    rng = np.random.default_rng(6)
    T, M, t1 = 100, 7, 43
    a = _rand_a(rng, T, M)
    e, gs, zi = rng.standard_normal(T), rng.standard_normal(T), rng.standard_normal(M)
    s = O.forward(a, e, zi)
    s_head = O.forward(a[:t1], e[:t1], zi)
    carry = s_head[::-1][:M]  # s(t1-1), ..., s(t1-M)
    s_tail = O.forward(a[t1:], e[t1:], carry)
    np.testing.assert_allclose(np.concatenate([s_head, s_tail]), s, rtol=1e-12, atol=1e-12)
    ge, ga, gzi = O.backward(a, s, gs, zi)
    ge_tail, ga_tail, gzi_tail = O.backward(a[t1:], s[t1:], gs[t1:], carry)
    np.testing.assert_allclose(ge_tail, ge[t1:], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ga_tail, ga[t1:], rtol=1e-12, atol=1e-12)
    # the tail's initial-state gradient is extra upstream gradient on s(t1-1..t1-M)
    gs_head = gs[:t1].copy()
    gs_head[::-1][:M] += gzi_tail
    ge_head, ga_head, gzi_head = O.backward(a[:t1], s[:t1], gs_head, zi)
    np.testing.assert_allclose(ge_head, ge[:t1], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(gzi_head, gzi, rtol=1e-10, atol=1e-12)


def test_batched_equals_per_signal():
    rng = np.random.default_rng(8)
    B, T, M = 3, 70, 4
    a = rng.uniform(-0.5, 0.5, (B, T, M))
    e, gs, zi = rng.standard_normal((B, T)), rng.standard_normal((B, T)), rng.standard_normal((B, M))
    s = O.forward(a, e, zi)
    ge, ga, gzi = O.backward(a, s, gs, zi)
    for b in range(B):
        assert np.array_equal(s[b], O.forward(a[b], e[b], zi[b]))
        g1 = O.backward(a[b], s[b], gs[b], zi[b])
        assert np.array_equal(ge[b], g1[0]) and np.array_equal(ga[b], g1[1]) and np.array_equal(gzi[b], g1[2])


def test_degenerate_shapes():
    s = O.forward(np.zeros((0, 3)), np.zeros(0))
    assert s.shape == (0,)
    # T < M: only the initial state and the first rows matter
    rng = np.random.default_rng(9)
    a = rng.uniform(-0.5, 0.5, (2, 6))
    e, zi = rng.standard_normal(2), rng.standard_normal(6)
    s = O.forward(a, e, zi)
    assert abs(s[0] - (e[0] - np.dot(a[0], zi))) < 1e-15
    assert abs(s[1] - (e[1] - a[1, 0] * s[0] - np.dot(a[1, 1:], zi[:5]))) < 1e-15
