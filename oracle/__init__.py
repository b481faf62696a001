"""Sequential FP64 oracle for the time-varying LP filter and its adjoint.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow statement of what
the CUDA library computes (Eq. 5, Eq. 11 and Eq. 12 of Yu & Fazekas,
arXiv 2406.05128).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import it.  The product path
(``paper_2406_05128_gb300``) never imports it and the two share no code.

The arithmetic lives in ``tvlp_oracle.c`` (plain C, double precision,
compiled here with gcc).  This module only marshals numpy arrays: inputs are
converted to float64 (exactly, from the float32 values the GPU sees) and
passed to the C routines one batch at a time.

Parity status of each routine (see the tests under ``tests/test_oracle_*``):
  forward   pinned: closed-form impulse responses, dense triangular solve,
            scipy.signal.lfilter, the IIR expansion of Eqs. 6-8, invariants.
  backward  pinned: dense transposed solve, finite differences, Eqs. 9-10,
            GOLF's time-invariant gradient (Eq. 3), adjoint identity.
  coeffs    pinned: the Levinson recursion of scipy.linalg.solve_toeplitz,
            the closed forms for M = 1, 2, frame anchors and midpoints,
            minimum phase (roots inside the unit circle).
  coeffs_adjoint  pinned: finite differences of <ga, a(k)> with respect to
            every frame coefficient, closed forms for M = 1, 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvlp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtvlp_oracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add, so the x86 and aarch64 builds
# round identically.
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off"]
LDLIBS = ["-lm"]


def build(force: bool = False) -> str:
    """Compile tvlp_oracle.c into oracle/_build/libtvlp_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, *LDLIBS], check=True)
        os.replace(tmp, _SO)
    return _SO


def load_library(path: str) -> ctypes.CDLL:
    """Open a compiled oracle (the real one or a test-built variant)."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.tvlp_oracle_forward_batch.argtypes = [i64, i64, ctypes.c_int, dp, dp, dp, dp]
    lib.tvlp_oracle_forward_batch.restype = None
    lib.tvlp_oracle_backward_batch.argtypes = [i64, i64, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp]
    lib.tvlp_oracle_backward_batch.restype = None
    lib.tvlp_oracle_coeffs_batch.argtypes = [i64, i64, ctypes.c_int, ctypes.c_int, dp, dp]
    lib.tvlp_oracle_coeffs_batch.restype = None
    lib.tvlp_oracle_coeffs_adjoint_batch.argtypes = [i64, i64, ctypes.c_int, ctypes.c_int, dp, dp, dp]
    lib.tvlp_oracle_coeffs_adjoint_batch.restype = None
    lib.tvlp_oracle_framewise_frames.argtypes = [i64, ctypes.c_int]
    lib.tvlp_oracle_framewise_frames.restype = i64
    lib.tvlp_oracle_framewise_batch.argtypes = [i64, i64, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp]
    lib.tvlp_oracle_framewise_batch.restype = None
    return lib


def _get():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _ptr(x):
    if x is None:
        return None
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float64)


def _batched(a, *vecs):
    """Promote single-signal arrays ([T,M], [T], [M]) to batch form."""
    single = a.ndim == 2
    if single:
        a = a[None]
        vecs = tuple(None if v is None else v[None] for v in vecs)
    return single, a, vecs


def forward(a, e, zi=None, lib=None):
    """Eq. 5: s(t) = e(t) - sum_i a_i(t) s(t-i).

    a: [B,T,M] (or [T,M]); e: [B,T]; zi: [B,M] with zi[...,j-1] = s(-j), or None.
    Returns s as float64 with the shape of e.
    """
    lib = lib or _get()
    a, e, zi = _f64(a), _f64(e), _f64(zi)
    single, a, (e, zi) = _batched(a, e, zi)
    B, T, M = a.shape
    assert e.shape == (B, T)
    assert zi is None or zi.shape == (B, M)
    s = np.empty((B, T), np.float64)
    lib.tvlp_oracle_forward_batch(B, T, M, _ptr(a), _ptr(e), _ptr(zi), _ptr(s))
    return s[0] if single else s


def backward(a, s, gs, zi=None, lib=None):
    """Eqs. 11-12 plus the initial-state gradient.

    Returns (ge [B,T], ga [B,T,M], gzi [B,M]) as float64.
    """
    lib = lib or _get()
    a, s, gs, zi = _f64(a), _f64(s), _f64(gs), _f64(zi)
    single, a, (s, gs, zi) = _batched(a, s, gs, zi)
    B, T, M = a.shape
    ge = np.empty((B, T), np.float64)
    ga = np.empty((B, T, M), np.float64)
    gzi = np.empty((B, M), np.float64)
    lib.tvlp_oracle_backward_batch(B, T, M, _ptr(a), _ptr(s), _ptr(zi), _ptr(gs),
                                   _ptr(ge), _ptr(ga), _ptr(gzi))
    if single:
        return ge[0], ga[0], gzi[0]
    return ge, ga, gzi


def forward_backward(a, e, gs, zi=None, lib=None):
    """One forward and one adjoint pass: returns (s, ge, ga, gzi)."""
    s = forward(a, e, zi, lib=lib)
    ge, ga, gzi = backward(a, s, gs, zi, lib=lib)
    return s, ge, ga, gzi


def n_frames(T: int, hop: int) -> int:
    """Frames of a T-sample signal at this hop: ceil(T / hop) + 1."""
    return -(-T // hop) + 1


def coeffs(k, T, hop, lib=None):
    """Sec. 4.3: per-sample direct-form coefficients a [B,T,M] (or [T,M])
    from frame-rate reflection coefficients k [B,F,M] (or [F,M]), F =
    ceil(T/hop)+1: linear interpolation, then the step-up recursion."""
    lib = lib or _get()
    k = _f64(k)
    single = k.ndim == 2
    if single:
        k = k[None]
    B, F, M = k.shape
    assert F == n_frames(T, hop), (F, T, hop)
    a = np.empty((B, T, M), np.float64)
    lib.tvlp_oracle_coeffs_batch(B, T, M, hop, _ptr(k), _ptr(a))
    return a[0] if single else a


def coeffs_adjoint(k, ga, hop, lib=None):
    """dL/dk [B,F,M] from dL/da [B,T,M] for the coefficients of coeffs()."""
    lib = lib or _get()
    k, ga = _f64(k), _f64(ga)
    single = k.ndim == 2
    if single:
        k, ga = k[None], ga[None]
    B, F, M = k.shape
    T = ga.shape[1]
    assert F == n_frames(T, hop) and ga.shape == (B, T, M)
    gk = np.empty((B, F, M), np.float64)
    lib.tvlp_oracle_coeffs_adjoint_batch(B, T, M, hop, _ptr(k), _ptr(ga), _ptr(gk))
    return gk[0] if single else gk


def framewise_frames(T: int, hop: int) -> int:
    """Frames of the frame-wise approximation: ceil(T / hop) + 3."""
    return -(-T // hop) + 3


def framewise(af, e, gs=None, hop=120, lib=None):
    """Frame-wise approximation of Eq. 5 with 75 % overlap-add (Sec. 3.2,
    Sec. 4) and, with gs, its adjoint.

    af: [B,F,M] direct-form coefficients per frame, F = framewise_frames(T, hop);
    e, gs: [B,T].  Returns s [B,T], or (s, ge [B,T], gaf [B,F,M]) with gs.
    """
    lib = lib or _get()
    af, e, gs = _f64(af), _f64(e), _f64(gs)
    B, F, M = af.shape
    T = e.shape[1]
    assert F == framewise_frames(T, hop) and e.shape == (B, T)
    s = np.empty((B, T), np.float64)
    ge = np.empty((B, T), np.float64) if gs is not None else None
    gaf = np.empty((B, F, M), np.float64) if gs is not None else None
    lib.tvlp_oracle_framewise_batch(B, T, M, hop, _ptr(af), _ptr(e), _ptr(gs), _ptr(s), _ptr(ge), _ptr(gaf))
    return s if gs is None else (s, ge, gaf)
