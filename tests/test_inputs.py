"""The seeded input generators: shapes, determinism and the properties the
workloads rely on (stable frozen filters, anchors of the interpolation)."""
import numpy as np

from paper_2406_05128_gb300 import inputs


def test_step_up_low_orders():
    k = np.array([[0.3], [-0.7]])
    np.testing.assert_allclose(inputs.step_up(k), k)
    k2 = np.array([0.4, -0.5])
    # order 2: a_1 = k_1 (1 + k_2), a_2 = k_2
    np.testing.assert_allclose(inputs.step_up(k2), [0.4 * 0.5, -0.5])


def test_step_up_is_minimum_phase():
    rng = np.random.default_rng(0)
    for M in (4, 16, 22, 30):
        k = rng.uniform(-0.95, 0.95, size=(20, M))
        a = inputs.step_up(k)
        for row in a:
            assert np.max(np.abs(np.roots(np.concatenate([[1.0], row])))) < 1.0


def test_step_up_inverts_levinson_step_down():
    """Step-down (backward Levinson) recovers the reflection coefficients."""
    rng = np.random.default_rng(1)
    M = 9
    k = rng.uniform(-0.9, 0.9, size=M)
    a = list(inputs.step_up(k))
    rec = []
    for m in range(M, 0, -1):
        km = a[m - 1]
        rec.append(km)
        a = [(a[i] - km * a[m - 2 - i]) / (1 - km * km) for i in range(m - 1)]
    np.testing.assert_allclose(rec[::-1], k, rtol=1e-12, atol=1e-12)


def test_upsampling_hits_anchors_and_is_linear():
    rng = np.random.default_rng(2)
    k = rng.standard_normal((2, 5, 3))
    kt = inputs.upsample_frames(k, 4 * 120, 120)
    np.testing.assert_allclose(kt[:, ::120], k[:, :4])
    np.testing.assert_allclose(kt[:, 60], 0.5 * (k[:, 0] + k[:, 1]))


def test_pulse_train_rate_and_determinism():
    p1 = inputs.pulse_train(np.random.default_rng(3), 4, 24000)
    p2 = inputs.pulse_train(np.random.default_rng(3), 4, 24000)
    assert np.array_equal(p1, p2)
    f0 = np.random.default_rng(3).uniform(100, 600, size=(4, 1))[:, 0]
    np.testing.assert_allclose(p1.sum(axis=1), f0, atol=1.0)


def test_workload_shapes_and_dtypes():
    w = inputs.make("t", 3, 500, 7, seed=4, with_zi=True)
    assert w.a.shape == (3, 500, 7) and w.a.dtype == np.float32
    assert w.e.shape == (3, 500) and w.gs.shape == (3, 500) and w.zi.shape == (3, 7)
    w2 = inputs.make("t", 3, 500, 7, seed=4, with_zi=True)
    assert np.array_equal(w.a, w2.a) and np.array_equal(w.e, w2.e)
