"""Shared test helpers: the parity metric and workload construction."""
from __future__ import annotations

import numpy as np

# Parity tolerance for FP32 results: max over samples of |gpu - oracle|
# divided by max |oracle|, per signal (and per output: s, ge, ga).
TOL_F32 = 1e-4
TOL_F64 = 1e-10


def norm_err(x, ref):
    """Per-signal normalised max error: max|x-ref| / max|ref| over all but
    the leading (signal) axis.  Returns an array of shape [B]."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    B = ref.shape[0]
    d = np.abs(x - ref).reshape(B, -1).max(axis=1) if ref.size else np.zeros(B)
    m = np.abs(ref).reshape(B, -1).max(axis=1) if ref.size else np.ones(B)
    return d / np.where(m > 0, m, 1.0)


def assert_close(name, x, ref, tol):
    err = norm_err(x, ref)
    worst = float(err.max()) if err.size else 0.0
    assert worst <= tol, f"{name}: normalised error {worst:.3e} > {tol:.0e} (per-signal {np.round(err, 9)})"
    return worst
