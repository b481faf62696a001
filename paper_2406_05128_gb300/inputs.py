"""Seeded synthetic inputs for the time-varying LP filter.

This module is shared by the tests, the benchmark and the smoke check; it
holds none of the filter's arithmetic.  It draws the signals the paper's
workloads are made of and turns frame-rate reflection coefficients into the
per-sample direct-form coefficients the filter consumes:

* reflection coefficients per frame (Sec. 4.3: the encoder emits reflection
  coefficients), drawn uniformly;
* linear upsampling of the frame values to the sample rate (Sec. 4.3);
* the step-up recursion from reflection to direct-form coefficients
  (the paper names the parameterisation but does not print the conversion);
* excitations: Gaussian noise and a pulse train standing in for the glottal
  wavetable source of Sec. 2.1;
* the upstream gradient dL/ds as Gaussian noise.

Everything is float64 internally and returned as float32, the storage type of
the CUDA path.  The same arrays feed the CUDA library and the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SAMPLE_RATE = 24000
HOP = 120


def reflection_frames(rng, B, F, M, kmax, decay=1.0):
    """k[b, f, m-1] ~ U(-kmax, kmax) * decay**(m-1): [B, F, M] float64."""
    k = rng.uniform(-kmax, kmax, size=(B, F, M))
    if decay != 1.0:
        k *= decay ** np.arange(M, dtype=np.float64)
    return k


def n_frames(T, hop=HOP):
    """Frames needed so that every sample lies between two anchors."""
    return int(math.ceil(T / hop)) + 1


def upsample_frames(k, T, hop=HOP):
    """Linear interpolation of frame values to samples.

    Frame f is anchored at sample f*hop; sample t lies between anchors
    floor(t/hop) and floor(t/hop)+1.  k: [B, F, M] -> [B, T, M].
    """
    t = np.arange(T)
    f = t // hop
    w = ((t - f * hop) / hop)[None, :, None]
    return k[:, f, :] * (1.0 - w) + k[:, f + 1, :] * w


def step_up(k):
    """Reflection coefficients -> direct-form coefficients, last axis.

    With A(z) = 1 + sum_i a_i z^-i:  a^(m)_m = k_m and
    a^(m)_i = a^(m-1)_i + k_m a^(m-1)_{m-i} for i < m.  Every |k_m| < 1
    gives a minimum-phase A(z), so each frozen filter is stable.
    """
    k = np.asarray(k, dtype=np.float64)
    M = k.shape[-1]
    a = np.zeros_like(k)
    for m in range(1, M + 1):
        km = k[..., m - 1:m]
        prev = a[..., : m - 1].copy()
        a[..., : m - 1] = prev + km * prev[..., ::-1]
        a[..., m - 1] = k[..., m - 1]
    return a


def pulse_train(rng, B, T, f0_lo=100.0, f0_hi=600.0, sr=SAMPLE_RATE):
    """Unit pulses at a per-signal constant F0 ~ U(f0_lo, f0_hi).

    A phase accumulator advances by F0/sr per sample and a pulse of 1.0 is
    emitted on the sample where it wraps.  Returns [B, T] float64.
    """
    f0 = rng.uniform(f0_lo, f0_hi, size=(B, 1))
    phase = np.cumsum(np.broadcast_to(f0 / sr, (B, T)), axis=1)
    wraps = np.floor(phase)
    prev = np.concatenate([np.zeros((B, 1)), wraps[:, :-1]], axis=1)
    return (wraps > prev).astype(np.float64)


def coefficients(rng, B, T, M, kmax, decay=1.0, hop=HOP):
    """Per-sample direct-form coefficients a [B, T, M] from frame-rate k."""
    k = reflection_frames(rng, B, n_frames(T, hop), M, kmax, decay)
    return step_up(upsample_frames(k, T, hop))


@dataclass
class Workload:
    """One seeded batch: a [B,T,M], e [B,T], gs [B,T] (float32), zi or None."""
    name: str
    a: np.ndarray
    e: np.ndarray
    gs: np.ndarray
    zi: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.a.shape


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


# Coefficient generators (see the design notes on conditioning):
#   "literal": k ~ U(-kmax, kmax) in every order (timing workloads);
#   "stable":  k_m ~ U(-0.95, 0.95) * 0.9**(m-1), speech-like decay of the
#              higher-order reflection coefficients (parity workloads).
def make(name, B, T, M, *, seed, kmax=0.95, gen="stable", excitation="noise",
         hop=HOP, with_zi=False):
    rng = np.random.default_rng(seed)
    decay = 0.9 if gen == "stable" else 1.0
    a = coefficients(rng, B, T, M, kmax, decay, hop)
    if excitation == "noise":
        e = rng.standard_normal((B, T))
    elif excitation == "pulse":
        e = pulse_train(rng, B, T) + 0.1 * rng.standard_normal((B, T))
    else:
        raise ValueError(excitation)
    gs = rng.standard_normal((B, T))
    zi = rng.standard_normal((B, M)) if with_zi else None
    return Workload(name, _f32(a), _f32(e), _f32(gs), None if zi is None else _f32(zi),
                    dict(B=B, T=T, M=M, seed=seed, kmax=kmax, gen=gen,
                         excitation=excitation, hop=hop))


def plain_small(seed=1, gen="literal"):
    """B=1, T=4800, M=16, k ~ U(-0.9, 0.9), e ~ N(0,1) (the small plain case)."""
    return make("plain B=1 T=4800 M=16", 1, 4800, 16, seed=seed, kmax=0.9,
                gen=gen, excitation="noise")


def batched_headline(seed=2, gen="literal", B=32, T=48000, M=22):
    """B=32, T=48000 (2 s at 24 kHz), M=22, pulse train + 0.1 N(0,1)."""
    return make(f"batched B={B} T={T} M={M}", B, T, M, seed=seed, kmax=0.95,
                gen=gen, excitation="pulse")


# ---------------------------------------------------------------------------
# The same recipe on the GPU, for workloads too large to draw on the host:
# frame-rate reflection coefficients from a seeded numpy generator, then
# linear upsampling and the step-up recursion as torch operations.  One
# signal per entry of `lengths`; returns lists of per-signal tensors.
# ---------------------------------------------------------------------------
def signals_torch(lengths, M, *, seed, kmax=0.95, gen="stable", hop=HOP, device="cuda"):
    """Per signal b of length T_b: a [T_b, M], e [T_b] (pulse train + 0.1
    N(0,1)), gs [T_b] ~ N(0,1), all float32 on `device`."""
    import torch

    rng = np.random.default_rng(seed)
    decay = 0.9 if gen == "stable" else 1.0
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = []
    for T in lengths:
        T = int(T)
        k = torch.tensor(reflection_frames(rng, 1, n_frames(max(T, 1), hop), M, kmax, decay)[0], device=device)
        t = torch.arange(T, device=device)
        f = torch.div(t, hop, rounding_mode="floor")
        w = ((t - f * hop).to(torch.float64) / hop)[:, None]
        kt = k[f] * (1.0 - w) + k[f + 1] * w  # [T, M] float64
        a = torch.zeros_like(kt)
        for m in range(1, M + 1):
            km = kt[:, m - 1:m]
            prev = a[:, : m - 1].clone()
            a[:, : m - 1] = prev + km * prev.flip(1)
            a[:, m - 1] = kt[:, m - 1]
        f0 = float(rng.uniform(100.0, 600.0))
        phase = torch.cumsum(torch.full((T,), f0 / SAMPLE_RATE, dtype=torch.float64, device=device), 0)
        wraps = torch.floor(phase)
        prev = torch.cat([torch.zeros(1, dtype=torch.float64, device=device), wraps[:-1]])
        e = (wraps > prev).to(torch.float64) + 0.1 * torch.randn(T, generator=g, dtype=torch.float64, device=device)
        gs = torch.randn(T, generator=g, dtype=torch.float64, device=device)
        out.append((a.float().contiguous(), e.float(), gs.float()))
    return out
