"""The frame-wise overlap-add approximation (the GOLF-ff comparison of
Sec. 4.3; per-frame time-invariant filters, 75 % overlap as in Sec. 5.2) through the C ABI
against its FP64 oracle: s, dL/de and the per-frame coefficient gradient,
per signal within 1e-4 of the oracle's scale."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2406_05128_gb300 import _lib, inputs, ops  # noqa: E402
from tests.helpers import TOL_F32, assert_close  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


def _workload(B, T, M, hop, seed, kmax=0.95, decay=0.9):
    """Stable reflection generator (per-order decay 0.9, as for the other
    parity workloads): with |k| up to 0.95 at every order, a frame's
    time-invariant filter at M >= 22 is resonant enough that FP32 direct-form
    filtering alone departs from FP64 by about 1e-3 over one frame."""
    rng = np.random.default_rng(seed)
    F = O.framewise_frames(T, hop)
    af = inputs.step_up(inputs.reflection_frames(rng, B, F, M, kmax, decay)).astype(np.float32)
    e = (inputs.pulse_train(rng, B, T) + 0.1 * rng.standard_normal((B, T))).astype(np.float32)
    gs = rng.standard_normal((B, T)).astype(np.float32)
    return af, e, gs


def _gpu(af, e, gs, hop):
    afd, ed, gsd = (torch.tensor(x, device=DEV) for x in (af, e, gs))
    s, y = ops.lp_framewise_forward(afd, ed, hop)
    ge, gaf = ops.lp_framewise_backward(gsd, afd, y, hop)
    torch.cuda.synchronize()
    return s.cpu().numpy(), ge.cpu().numpy(), gaf.cpu().numpy()


@pytest.mark.parametrize("B,T,M,hop", [(2, 1000, 4, 8), (3, 1237, 16, 120), (2, 5000, 22, 120), (1, 777, 30, 64),
                                       (2, 2400, 32, 120), (2, 130, 1, 16), (1, 5, 22, 120), (2, 960, 12, 512)])
def test_framewise_matches_oracle(B, T, M, hop):
    af, e, gs = _workload(B, T, M, hop, seed=T + M)
    s, ge, gaf = _gpu(af, e, gs, hop)
    rs, rge, rgaf = O.framewise(af, e, gs, hop=hop)
    assert_close("s", s, rs, TOL_F32)
    assert_close("ge", ge, rge, TOL_F32)
    assert_close("gaf", gaf, rgaf, TOL_F32)


def test_framewise_headline_shape():
    """B=32, T=48000, M=22, hop 120 (the headline shape), every output."""
    af, e, gs = _workload(32, 48000, 22, 120, seed=2)
    s, ge, gaf = _gpu(af, e, gs, 120)
    rs, rge, rgaf = O.framewise(af, e, gs, hop=120)
    print("framewise headline errors",
          assert_close("s", s, rs, TOL_F32), assert_close("ge", ge, rge, TOL_F32),
          assert_close("gaf", gaf, rgaf, TOL_F32))


def test_framewise_zero_order_is_identity():
    rng = np.random.default_rng(1)
    T, hop = 3000, 120
    e = torch.tensor(rng.standard_normal((2, T)).astype(np.float32), device=DEV)
    af = torch.zeros((2, ops.framewise_frames(T, hop), 0), device=DEV)
    s, _ = ops.lp_framewise_forward(af, e, hop)
    torch.cuda.synchronize()
    assert torch.allclose(s, e, atol=1e-6, rtol=0)


def test_framewise_autograd():
    af, e, gs = _workload(2, 3000, 8, 120, seed=9)
    afd = torch.tensor(af, device=DEV, requires_grad=True)
    ed = torch.tensor(e, device=DEV, requires_grad=True)
    s = ops.lp_filter_framewise(afd, ed, 120)
    s.backward(torch.tensor(gs, device=DEV))
    rs, rge, rgaf = O.framewise(af, e, gs, hop=120)
    assert_close("s", s.detach().cpu().numpy(), rs, TOL_F32)
    assert_close("ge", ed.grad.cpu().numpy(), rge, TOL_F32)
    assert_close("gaf", afd.grad.cpu().numpy(), rgaf, TOL_F32)


def test_framewise_invalid_arguments():
    e = torch.zeros((1, 100), device=DEV)
    for hop in (0, 12, 1024):
        af = torch.zeros((1, max(ops.framewise_frames(100, max(hop, 1)), 1), 4), device=DEV)
        with pytest.raises(_lib.LPError):
            _lib.lp_framewise_forward(1, 100, 4, hop, af.data_ptr(), e.data_ptr(), e.data_ptr(), None,
                                      torch.cuda.current_stream().cuda_stream)
