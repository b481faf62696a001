"""Source-filter synthesis (Eq. 4, S = (G + N C) H) with synthetic
parameters, differentiated end to end.

    e(t) = g(t) (pulse(t) + (noise * c)(t)),   s = LP_{a(t)}(e)

g(t) is a per-sample gain interpolated from frame gains, c a per-signal FIR
applied to white noise, and a(t) the coefficients the kernels generate from
reflection coefficients per frame.  H is the proposed filter with its input
gain.  The gradients of <s, w> with respect to the frame gains, the FIR
taps and the reflection coefficients, computed through the library's
autograd op, must match a float64 reference.  The reference runs the
filter and its adjoint in the oracle, the coefficient gradient through the
oracle's chain rule, and the gain and FIR in float64 torch on the CPU.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2406_05128_gb300 import _lib, inputs, ops  # noqa: E402
from tests.helpers import TOL_F32  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


def frame_interp(x, T, hop):
    """x [B, F] per frame -> [B, T] per sample: frame f at sample f*hop,
    linear in between (the same anchoring as the coefficients)."""
    t = torch.arange(T, device=x.device)
    f = torch.div(t, hop, rounding_mode="floor")
    w = ((t - f * hop).to(x.dtype) / hop)[None]
    return x[:, f] * (1 - w) + x[:, f + 1] * w


def excitation(gain_frames, c, pulse, noise, hop):
    """e = g (pulse + noise * c), with a causal per-signal FIR."""
    B, T = pulse.shape
    K = c.shape[1]
    filt = torch.nn.functional.conv1d(torch.nn.functional.pad(noise[None], (K - 1, 0)), c.flip(1)[:, None],
                                      groups=B)[0]
    return frame_interp(gain_frames, T, hop) * (pulse + filt)


def test_golf_ss_gradients_match_float64_reference():
    B, T, M, hop, K = 2, 4800, 22, 120, 33
    rng = np.random.default_rng(12)
    F = ops.n_frames(T, hop)
    k = inputs.reflection_frames(rng, B, F, M, 0.95, 0.9).astype(np.float32)
    gain = (0.5 + rng.random((B, F))).astype(np.float32)
    c = (0.1 * rng.standard_normal((B, K))).astype(np.float32)
    pulse = inputs.pulse_train(rng, B, T).astype(np.float32)
    noise = rng.standard_normal((B, T)).astype(np.float32)
    wgt = rng.standard_normal((B, T)).astype(np.float32)

    # the library: autograd through ops.lp_filter_frames on the GPU
    kt = torch.tensor(k, device=DEV, requires_grad=True)
    gt = torch.tensor(gain, device=DEV, requires_grad=True)
    ct = torch.tensor(c, device=DEV, requires_grad=True)
    e = excitation(gt, ct, torch.tensor(pulse, device=DEV), torch.tensor(noise, device=DEV), hop)
    s = ops.lp_filter_frames(kt, e, hop)
    (s * torch.tensor(wgt, device=DEV)).sum().backward()
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0

    # float64 reference: the oracle for H, float64 torch on the CPU for the rest
    g64 = torch.tensor(gain, dtype=torch.float64, requires_grad=True)
    c64 = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    e64 = excitation(g64, c64, torch.tensor(pulse, dtype=torch.float64), torch.tensor(noise, dtype=torch.float64),
                     hop)
    a = O.coeffs(k, T, hop)
    rs = O.forward(a, e64.detach().numpy())
    rge, rga, _ = O.backward(a, rs, wgt.astype(np.float64))
    e64.backward(torch.tensor(rge))
    rgk = O.coeffs_adjoint(k, rga, hop)

    def close(name, got, ref):
        got, ref = np.asarray(got, np.float64).reshape(B, -1), np.asarray(ref, np.float64).reshape(B, -1)
        err = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
        assert err.max() <= TOL_F32, (name, err)

    close("s", s.detach().cpu().numpy(), rs)
    close("dL/dgain", gt.grad.cpu().numpy(), g64.grad.numpy())
    close("dL/dc", ct.grad.cpu().numpy(), c64.grad.numpy())
    close("dL/dk", kt.grad.cpu().numpy(), rgk)
