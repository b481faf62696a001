"""Chunk-state checkpointing: the backward recomputes s from the forward's
per-chunk incoming states (lp_tv_backward_recompute_*), and the autograd op
with checkpoint=True, against the FP64 oracle.

The differentiation workload is the harmonic-plus-noise synthesis
s = LP_{a_H}(pulse train) + LP_{a_C}(N(0,1)) with a multi-resolution STFT L1
loss (FFT sizes 509, 1021, 2053 as in the paper's training setup), run at a
size the oracle checks in seconds.
"""
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


def _tensors(w, dtype=torch.float32):
    a = torch.tensor(w.a, dtype=dtype, device=DEV)
    e = torch.tensor(w.e, dtype=dtype, device=DEV)
    gs = torch.tensor(w.gs, dtype=dtype, device=DEV)
    zi = torch.tensor(w.zi, dtype=dtype, device=DEV) if w.zi is not None else None
    return a, e, gs, zi


@pytest.mark.parametrize("B,T,M,chunk,zi", [(3, 5000, 22, 0, True), (2, 1237, 16, 48, False), (4, 3000, 30, 0, True)])
def test_recompute_backward_matches_oracle(B, T, M, chunk, zi):
    w = inputs.make("ck", B, T, M, seed=100 + T, gen="stable", with_zi=zi)
    a, e, gs, z = _tensors(w)
    s, ck = ops.lp_tv_forward(a, e, z, chunk=chunk, ckpt=True)
    ge, ga, gzi = ops.lp_tv_backward_recompute(gs, a, e, ck, z, need_gzi=zi, chunk=chunk)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    rs, rge, rga, rgzi = O.forward_backward(w.a, w.e, w.gs, w.zi)
    assert_close("ge", ge.cpu().numpy(), rge, TOL_F32)
    assert_close("ga", ga.cpu().numpy(), rga, TOL_F32)
    if zi:
        d = np.abs(gzi.cpu().numpy() - rgzi).max(axis=1) / np.abs(rge).max(axis=1)
        assert d.max() <= TOL_F32
    # the same adjoint from the stored s gives the same numbers: s is
    # recomputed bit for bit
    ge2, ga2, _ = ops.lp_tv_backward(gs, a, s, z, need_gzi=False, chunk=chunk)
    assert torch.equal(ge, ge2) and torch.equal(ga, ga2)


def test_recompute_rebuilds_s_bitwise():
    w = inputs.make("ckb", 2, 4000, 22, seed=7, gen="stable", with_zi=True)
    a, e, gs, z = _tensors(w)
    s, ck = ops.lp_tv_forward(a, e, z, ckpt=True)
    chunk = _lib.lp_tv_pick_chunk(2, 4000, 22)
    B, T, M = a.shape
    s2 = torch.full_like(s, float("nan"))
    ge = torch.empty_like(s)
    ws = ops.workspace(B, T, M, chunk, a.dtype, a.device)
    _lib.lp_tv_backward_recompute(_lib.LP_DTYPE_F32, B, T, M, gs.data_ptr(), a.data_ptr(), e.data_ptr(),
                                  ck.data_ptr(), z.data_ptr(), s2.data_ptr(), ge.data_ptr(), None, None, chunk, 0,
                                  ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.equal(s, s2)


def test_recompute_bitwise_with_defect_correction():
    """Resonant signals (literal generator, |k| <= 0.8) make the forward
    re-run part of its chunks from corrected states; the checkpoints keep
    those corrected states, so the recomputed s is still the forward's, bit
    for bit, and the adjoint from it meets the oracle."""
    w = inputs.make("ckl", 4, 48000, 22, seed=5, kmax=0.8, gen="literal", excitation="pulse")
    a, e, gs, _ = _tensors(w)
    s, ck = ops.lp_tv_forward(a, e, None, ckpt=True)
    ge, ga, _ = ops.lp_tv_backward_recompute(gs, a, e, ck, None, need_gzi=False)
    B, T, M = a.shape
    chunk = _lib.lp_tv_pick_chunk(B, T, M)
    s2 = torch.full_like(s, float("nan"))
    ge2 = torch.empty_like(s)
    ws = ops.workspace(B, T, M, chunk, a.dtype, a.device)
    _lib.lp_tv_backward_recompute(_lib.LP_DTYPE_F32, B, T, M, gs.data_ptr(), a.data_ptr(), e.data_ptr(),
                                  ck.data_ptr(), None, s2.data_ptr(), ge2.data_ptr(), None, None, chunk, 0,
                                  ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    assert torch.equal(s, s2)
    rs, rge, rga, _ = O.forward_backward(w.a, w.e, w.gs, None)
    assert_close("s", s.cpu().numpy(), rs, TOL_F32)
    assert_close("ge", ge.cpu().numpy(), rge, TOL_F32)
    assert_close("ga", ga.cpu().numpy(), rga, TOL_F32)


def test_gradcheck_f64_checkpointed():
    """torch.autograd.gradcheck in FP64 at B=2, T=256, M=4 with chunk-state
    checkpointing on (several chunks)."""
    w = inputs.make("gck", 2, 256, 4, seed=3, gen="stable", with_zi=True)
    a = torch.tensor(w.a, dtype=torch.float64, device=DEV, requires_grad=True)
    e = torch.tensor(w.e, dtype=torch.float64, device=DEV, requires_grad=True)
    zi = torch.tensor(w.zi, dtype=torch.float64, device=DEV, requires_grad=True)
    fn = lambda a_, e_, z_: ops.lp_filter(a_, e_, z_, chunk=32, checkpoint=True)
    assert torch.autograd.gradcheck(fn, (a, e, zi), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_checkpointed_autograd_matches_default_and_oracle():
    w = inputs.make("cka", 3, 6000, 22, seed=12, gen="stable", with_zi=True)
    grads = []
    for checkpoint in (False, True):
        a = torch.tensor(w.a, device=DEV, requires_grad=True)
        e = torch.tensor(w.e, device=DEV, requires_grad=True)
        zi = torch.tensor(w.zi, device=DEV, requires_grad=True)
        s = ops.lp_filter(a, e, zi, checkpoint=checkpoint)
        s.backward(torch.tensor(w.gs, device=DEV))
        grads.append([x.detach().cpu().numpy() for x in (s, e.grad, a.grad, zi.grad)])
    rs, rge, rga, rgzi = O.forward_backward(w.a, w.e, w.gs, w.zi)
    for g in grads:
        assert_close("s", g[0], rs, TOL_F32)
        assert_close("ge", g[1], rge, TOL_F32)
        assert_close("ga", g[2], rga, TOL_F32)
    assert np.array_equal(grads[0][0], grads[1][0])


def test_checkpoint_keeps_less_than_s():
    """What the autograd graph keeps for the backward beyond the inputs:
    s and the workspace by default, only the chunk checkpoints (M values per
    chunk) with checkpoint=True."""
    B, T, M = 2, 48000, 22
    a = torch.zeros((B, T, M), device=DEV, requires_grad=True)
    e = torch.randn((B, T), device=DEV, requires_grad=True)
    input_ptrs = {a.data_ptr(), e.data_ptr()}

    def extra_bytes(checkpoint):
        saved = []

        def pack(t):
            if t.data_ptr() not in input_ptrs:
                saved.append(t.numel() * t.element_size())
            return t

        with torch.autograd.graph.saved_tensors_hooks(pack, lambda t: t):
            s = ops.lp_filter(a, e, checkpoint=checkpoint)
        del s
        return sum(saved)

    full, ck = extra_bytes(False), extra_bytes(True)
    nC = _lib.lp_tv_num_chunks(T, M, _lib.lp_tv_pick_chunk(B, T, M))
    assert ck == B * nC * M * 4
    assert full >= B * T * 4 + _lib.lp_tv_workspace_bytes(B, T, M, 0)
    assert ck * 10 < full, (ck, full)


def _mss_loss(x, y, sizes=(509, 1021, 2053)):
    """Multi-resolution STFT L1 loss: L1 of linear and of log magnitudes,
    Hann windows, hop n_fft/4 (the paper gives only the FFT sizes)."""
    loss = 0.0
    for n in sizes:
        win = torch.hann_window(n, device=x.device, dtype=x.dtype)
        X = torch.stft(x, n, hop_length=n // 4, window=win, return_complex=True).abs()
        Y = torch.stft(y, n, hop_length=n // 4, window=win, return_complex=True).abs()
        loss = loss + (X - Y).abs().mean() + (torch.log(X + 1e-5) - torch.log(Y + 1e-5)).abs().mean()
    return loss


def test_harmonic_plus_noise_training_step():
    """s = LP_{a_H}(pulse) + LP_{a_C}(noise), both M=22 time-varying, MSS
    loss against a fixed target; the checkpointed training step gives the
    gradients of the default one and of the FP64 oracle's adjoint driven by
    the same dL/ds."""
    B, T, M = 4, 9600, 22
    wh = inputs.make("hn_h", B, T, M, seed=21, gen="stable", excitation="pulse")
    wc = inputs.make("hn_c", B, T, M, seed=22, gen="stable", excitation="noise")
    wt = inputs.make("hn_t", B, T, M, seed=23, gen="stable", excitation="pulse")
    target = torch.tensor(wt.e, device=DEV)
    results = []
    for checkpoint in (False, True):
        aH = torch.tensor(wh.a, device=DEV, requires_grad=True)
        aC = torch.tensor(wc.a, device=DEV, requires_grad=True)
        eH = torch.tensor(wh.e, device=DEV)
        eC = torch.tensor(wc.e, device=DEV)
        sH = ops.lp_filter(aH, eH, checkpoint=checkpoint)
        sC = ops.lp_filter(aC, eC, checkpoint=checkpoint)
        s = sH + sC
        s.retain_grad()
        loss = _mss_loss(s, target)
        loss.backward()
        results.append((s.detach().cpu().numpy(), s.grad.detach().cpu().numpy(), aH.grad.cpu().numpy(),
                        aC.grad.cpu().numpy()))
    (s0, g0, gaH0, gaC0), (s1, g1, gaH1, gaC1) = results
    assert np.array_equal(s0, s1)
    # the oracle's adjoint with the loss gradient as dL/ds
    gs = g0.astype(np.float32)
    _, _, rgaH, _ = O.forward_backward(wh.a, wh.e, gs)
    _, _, rgaC, _ = O.forward_backward(wc.a, wc.e, gs)
    for gaH, gaC in ((gaH0, gaC0), (gaH1, gaC1)):
        assert_close("ga_H", gaH, rgaH, TOL_F32)
        assert_close("ga_C", gaC, rgaC, TOL_F32)


def test_training_shape_full_size_sampled():
    """The differentiation workload at full size: B=64, T=96000, two M=22
    filters through the checkpointed autograd op (the bench's launch
    configuration); two signals of each filter against the oracle."""
    B, T, M = 64, 96000, 22
    sig_h = inputs.signals_torch([T] * B, M, seed=21, gen="stable", device=DEV)
    sig_c = inputs.signals_torch([T] * B, M, seed=22, gen="stable", device=DEV)
    aH = torch.stack([x[0] for x in sig_h]).requires_grad_(True)
    aC = torch.stack([x[0] for x in sig_c]).requires_grad_(True)
    eH = torch.stack([x[1] for x in sig_h])
    eC = torch.stack([x[2] for x in sig_c])  # an N(0,1) excitation
    g = torch.stack([x[2] for x in sig_h])
    sH = ops.lp_filter(aH, eH, checkpoint=True)
    sC = ops.lp_filter(aC, eC, checkpoint=True)
    (sH + sC).backward(g)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    for a, e, s, ga in ((aH, eH, sH, aH.grad), (aC, eC, sC, aC.grad)):
        for b in (0, B - 1):
            an, en, gn = (x[b].detach().cpu().numpy()[None] for x in (a, e, g))
            rs, rge, rga, _ = O.forward_backward(an, en, gn)
            assert_close("s", s[b].detach().cpu().numpy()[None], rs, TOL_F32)
            assert_close("ga", ga[b].cpu().numpy()[None], rga, TOL_F32)
