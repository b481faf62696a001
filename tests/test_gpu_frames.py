"""Coefficients generated in the kernels, against the FP64 oracle.

Frames (Sec. 4.3 moved onto the GPU): k [B, F, M] reflection coefficients
per frame, interpolated per sample and stepped up to a(t) inside every pass.
The oracle computes a(t) = coeffs(k) in FP64, runs Eq. 5 / Eqs. 11-12 on it,
and takes dL/da back to dL/dk with coeffs_adjoint.  Time-invariant (Eq. 2):
a [B, M]; the oracle broadcasts it over time and sums Eq. 12 over t (Eq. 3).
Tolerance: the FP32 bound of the other parity tests, per signal, normalised
by the largest reference value (gk per signal over all frames and orders).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2406_05128_gb300 import _lib, inputs, ops  # noqa: E402
from tests.helpers import TOL_F32, norm_err  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


def _case(B, T, M, hop, seed, zi=True):
    rng = np.random.default_rng(seed)
    k = inputs.reflection_frames(rng, B, O.n_frames(T, hop), M, 0.95, 0.9).astype(np.float32)
    e = inputs.pulse_train(rng, B, T).astype(np.float32) + 0.1 * rng.standard_normal((B, T)).astype(np.float32)
    gs = rng.standard_normal((B, T)).astype(np.float32)
    z = (0.1 * rng.standard_normal((B, M))).astype(np.float32) if zi else None
    return k, e, gs, z


def _t(x):
    return None if x is None else torch.tensor(x, device=DEV)


def _close(name, got, ref, tol=TOL_F32):
    got = np.asarray(got, np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    err = norm_err(got, ref)
    assert err.max() <= tol, (name, err)
    return err.max()


CASES = [
    # B, T, M, hop, chunk
    (2, 5000, 22, 120, 0),
    (3, 1237, 16, 120, 0),     # ragged tail, T not a multiple of hop
    (2, 2400, 22, 120, 48),    # T a multiple of hop, short chunks
    (2, 3001, 30, 80, 0),
    (2, 999, 13, 7, 0),        # padded order, short hop
    (1, 50, 8, 120, 0),        # T < hop
    (4, 777, 4, 33, 32),
]


@pytest.mark.parametrize("B,T,M,hop,chunk", CASES)
@pytest.mark.parametrize("reuse", [True, False])
def test_frames_match_oracle(B, T, M, hop, chunk, reuse):
    k, e, gs, zi = _case(B, T, M, hop, seed=B * 7 + T + M)
    kt, et, gst, zit = _t(k), _t(e), _t(gs), _t(zi)
    ws = ops.workspace_frames(B, T, M, hop, chunk, DEV)
    s = ops.lp_tv_forward_frames(kt, et, hop, zit, chunk=chunk, ws=ws)
    ge, gk, gzi = ops.lp_tv_backward_frames(gst, kt, s, hop, zit, chunk=chunk, ws=ws, reuse_forward=reuse)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    a = O.coeffs(k, T, hop)
    rs, rge, rga, rgzi = O.forward_backward(a, e, gs, zi)
    rgk = O.coeffs_adjoint(k, rga, hop)
    _close("s", s.cpu().numpy(), rs)
    _close("ge", ge.cpu().numpy(), rge)
    _close("gk", gk.cpu().numpy(), rgk)
    d = np.abs(gzi.cpu().numpy() - rgzi).max(axis=1) / np.abs(rge).max(axis=1)
    assert d.max() <= TOL_F32


@pytest.mark.parametrize("B,T,M,hop,chunk", CASES)
@pytest.mark.parametrize("reuse", [True, False])
def test_frames_row_cache_same_bits(B, T, M, hop, chunk, reuse):
    """With the cached workspace, the forward's first pass keeps every
    generated row and the later passes stream them: the same bits as
    generating them in every pass, and the kept rows are the oracle's a(t)."""
    k, e, gs, zi = _case(B, T, M, hop, seed=B * 5 + T + M)
    kt, et, gst, zit = _t(k), _t(e), _t(gs), _t(zi)
    got = []
    for cache in (False, True):
        ws = ops.workspace_frames(B, T, M, hop, chunk, DEV, cache_rows=cache)
        s = ops.lp_tv_forward_frames(kt, et, hop, zit, chunk=chunk, ws=ws)
        ge, gk, gzi = ops.lp_tv_backward_frames(gst, kt, s, hop, zit, chunk=chunk, ws=ws, reuse_forward=reuse)
        torch.cuda.synchronize()
        assert _lib.lp_tv_device_status() == 0
        got.append([x.cpu().numpy() for x in (s, ge, gk, gzi)])
        if cache:
            n0 = _lib.lp_tv_workspace_bytes_frames(B, T, M, hop, chunk)
            n1 = _lib.lp_tv_workspace_bytes_frames_cached(B, T, M, hop, chunk)
            if M in (2, 4, 8, 12, 16, 22, 30, 32):
                assert n1 >= n0 + B * T * M * 4
                rows = ws[n0:n0 + B * T * M * 4].view(torch.float32).reshape(B, T, M).cpu().numpy()
                ref = O.coeffs(k, T, hop)
                err = np.abs(rows - ref).max() / max(np.abs(ref).max(), 1e-30)
                assert err <= TOL_F32, err
            else:
                assert n1 == n0  # padded orders keep no cache
    for x, y in zip(*got):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))


def test_frames_headline_shape():
    """B=32, T=48000, M=22, hop 120, with the row cache: every sample of s
    and ge, and every frame gradient of two signals, against the oracle."""
    B, T, M, hop = 32, 48000, 22, 120
    k, e, gs, _ = _case(B, T, M, hop, seed=2, zi=False)
    kt, et, gst = _t(k), _t(e), _t(gs)
    ws = ops.workspace_frames(B, T, M, hop, 0, DEV, cache_rows=True)
    s = ops.lp_tv_forward_frames(kt, et, hop, chunk=0, ws=ws)
    ge, gk, _ = ops.lp_tv_backward_frames(gst, kt, s, hop, need_gzi=False, ws=ws, reuse_forward=True)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    a = O.coeffs(k, T, hop)
    rs, rge, rga, _ = O.forward_backward(a, e, gs)
    # the oracle's dL/dk is O(M^3) per sample: two signals
    sel = [0, B - 1]
    rgk = O.coeffs_adjoint(k[sel], rga[sel], hop)
    print("frames headline errors", _close("s", s.cpu().numpy(), rs), _close("ge", ge.cpu().numpy(), rge),
          _close("gk", gk.cpu().numpy()[sel], rgk))


def test_frames_autograd_and_determinism():
    B, T, M, hop = 2, 3000, 22, 120
    k, e, gs, zi = _case(B, T, M, hop, seed=9)
    grads = []
    for _ in range(2):
        kt = _t(k).requires_grad_(True)
        et = _t(e).requires_grad_(True)
        zit = _t(zi).requires_grad_(True)
        s = ops.lp_filter_frames(kt, et, hop, zit)
        s.backward(_t(gs))
        grads.append([x.detach().cpu().numpy() for x in (s, kt.grad, et.grad, zit.grad)])
    for x, y in zip(*grads):
        assert np.array_equal(x, y)
    a = O.coeffs(k, T, hop)
    rs, rge, rga, rgzi = O.forward_backward(a, e, gs, zi)
    _close("s", grads[0][0], rs)
    _close("gk", grads[0][1], O.coeffs_adjoint(k, rga, hop))
    _close("ge", grads[0][2], rge)


def test_frames_varlen_forward():
    M, hop = 22, 120
    lengths = [5000, 17, 1, 2400, 999, 240]
    rng = np.random.default_rng(31)
    pk = ops.Packed(lengths, DEV)
    pf = ops.PackedFrames(pk, hop)
    ks = [inputs.reflection_frames(rng, 1, O.n_frames(n, hop), M, 0.95, 0.9)[0].astype(np.float32) for n in lengths]
    es = [rng.standard_normal(n).astype(np.float32) for n in lengths]
    k = pf.pack([_t(x) for x in ks])
    e = pk.pack([_t(x) for x in es])
    s = ops.lp_tv_forward_frames_varlen(pk, pf, k, e, chunk=96)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    for n, kk, ee, got in zip(lengths, ks, es, pk.unpack(s)):
        rs = O.forward(O.coeffs(kk, n, hop), ee)
        _close("s", got.cpu().numpy()[None], rs[None])
    # a signal alone gives the same bits as in the mix (fixed chunk)
    pk1 = ops.Packed([lengths[0]], DEV)
    pf1 = ops.PackedFrames(pk1, hop)
    s1 = ops.lp_tv_forward_frames_varlen(pk1, pf1, pf1.pack([_t(ks[0])]), pk1.pack([_t(es[0])]), chunk=96)
    assert torch.equal(s1[:lengths[0]], pk.unpack(s)[0])


@pytest.mark.parametrize("B,T,M,chunk", [(3, 5000, 22, 0), (2, 1237, 16, 48), (2, 700, 5, 0)])
def test_time_invariant_matches_oracle(B, T, M, chunk):
    rng = np.random.default_rng(T + M)
    kc = inputs.reflection_frames(rng, B, 1, M, 0.95, 0.9)[:, 0]
    a = np.stack([O.coeffs(np.stack([kc[b], kc[b]]), 1, 1)[0] for b in range(B)]).astype(np.float32)  # stable
    e = rng.standard_normal((B, T)).astype(np.float32)
    gs = rng.standard_normal((B, T)).astype(np.float32)
    zi = (0.1 * rng.standard_normal((B, M))).astype(np.float32)
    at, et, gst, zit = _t(a), _t(e), _t(gs), _t(zi)
    ws = ops.workspace_ti(B, T, M, chunk, DEV)
    s = ops.lp_tv_forward_ti(at, et, zit, chunk=chunk, ws=ws)
    ge, ga, gzi = ops.lp_tv_backward_ti(gst, at, s, zit, chunk=chunk, ws=ws, reuse_forward=True)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    abig = np.repeat(a[:, None, :], T, axis=1)
    rs, rge, rga, rgzi = O.forward_backward(abig, e, gs, zi)
    _close("s", s.cpu().numpy(), rs)
    _close("ge", ge.cpu().numpy(), rge)
    _close("ga", ga.cpu().numpy(), rga.sum(axis=1))
    # autograd front end gives the same numbers
    at2 = _t(a).requires_grad_(True)
    s2 = ops.lp_filter_ti(at2, et, zit, chunk=chunk)
    s2.backward(gst)
    assert torch.equal(s2.detach(), s) and torch.equal(at2.grad, ga)


def test_generated_degenerate_shapes():
    k = torch.zeros((2, ops.n_frames(0, 120), 4), device=DEV)
    e = torch.zeros((2, 0), device=DEV)
    s = ops.lp_tv_forward_frames(k, e, 120)
    ge, gk, gzi = ops.lp_tv_backward_frames(e, k, s, 120, torch.zeros((2, 4), device=DEV))
    assert s.shape == (2, 0) and torch.all(gk == 0) and torch.all(gzi == 0)
    # zero reflection coefficients: the identity filter
    T = 500
    k = torch.zeros((2, ops.n_frames(T, 120), 6), device=DEV)
    e = torch.randn((2, T), device=DEV)
    s = ops.lp_tv_forward_frames(k, e, 120)
    assert torch.equal(s, e)
    with pytest.raises(_lib.LPError):
        _lib.lp_tv_forward_frames(2, T, 6, 0, k.data_ptr(), e.data_ptr(), None, s.data_ptr(), None, 0, None, 0, None)


@pytest.mark.parametrize("reuse", [True, False])
def test_frames_varlen_backward_matches_oracle(reuse):
    """Varlen adjoint with generated coefficients: ge, gzi and dL/dk per
    signal against the oracle; the padded slot's extra frame gets no
    gradient beyond what the oracle gives the signal's own frames."""
    M, hop, chunk = 22, 120, 96
    lengths = [5000, 17, 1, 2400, 999, 240, 0, 3601]
    rng = np.random.default_rng(41)
    pk = ops.Packed(lengths, DEV)
    pf = ops.PackedFrames(pk, hop)
    ks = [inputs.reflection_frames(rng, 1, O.n_frames(n, hop), M, 0.95, 0.9)[0].astype(np.float32) for n in lengths]
    es = [rng.standard_normal(n).astype(np.float32) for n in lengths]
    gss = [rng.standard_normal(n).astype(np.float32) for n in lengths]
    zis = (0.1 * rng.standard_normal((len(lengths), M))).astype(np.float32)
    k = pf.pack([_t(x) for x in ks])
    e, gs = pk.pack([_t(x) for x in es]), pk.pack([_t(x) for x in gss])
    zi = _t(zis)
    nb = _lib.lp_tv_workspace_bytes_frames_varlen(pk.n, pk.total, M, pf.total, chunk)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
    s = ops.lp_tv_forward_frames_varlen(pk, pf, k, e, zi, chunk=chunk, ws=ws)
    ge, gk, gzi = ops.lp_tv_backward_frames_varlen(pk, pf, gs, k, s, zi, chunk=chunk, ws=ws, reuse_forward=reuse)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    ge_u, s_u = pk.unpack(ge), pk.unpack(s)
    for b, n in enumerate(lengths):
        fb, cnt = pf.starts[b], ops.n_frames(n, hop)
        gkb = gk[fb:fb + cnt].cpu().numpy()
        if n == 0:
            assert np.all(gkb == 0) and np.all(gzi[b].cpu().numpy() == 0)
            continue
        a = O.coeffs(ks[b], n, hop)
        rs, rge, rga, rgzi = O.forward_backward(a[None], es[b][None], gss[b][None], zis[b][None])
        rgk = O.coeffs_adjoint(ks[b], rga[0], hop)
        _close("s", s_u[b].cpu().numpy()[None], rs)
        _close("ge", ge_u[b].cpu().numpy()[None], rge)
        _close("gk", gkb[None], rgk[None])
        d = np.abs(gzi[b].cpu().numpy() - rgzi[0]).max() / np.abs(rge).max()
        assert d <= TOL_F32


@pytest.mark.parametrize("M", [22, 13])
def test_frames_varlen_row_cache_same_bits(M):
    """Varlen frames with the cached workspace: the forward keeps its rows
    and the adjoint (reusing the forward) streams them; the same bits as the
    uncached workspace, and the kept rows are the oracle's a(t).  M=13 is a
    padded order: no cache, the same workspace size."""
    hop, chunk = 120, 96
    lengths = [5000, 17, 1, 2400, 999, 240, 0, 3601]
    rng = np.random.default_rng(43)
    pk = ops.Packed(lengths, DEV)
    pf = ops.PackedFrames(pk, hop)
    ks = [inputs.reflection_frames(rng, 1, O.n_frames(n, hop), M, 0.95, 0.9)[0].astype(np.float32) for n in lengths]
    k = pf.pack([_t(x) for x in ks])
    e = pk.pack([_t(rng.standard_normal(n).astype(np.float32)) for n in lengths])
    gs = pk.pack([_t(rng.standard_normal(n).astype(np.float32)) for n in lengths])
    zi = _t((0.1 * rng.standard_normal((len(lengths), M))).astype(np.float32))
    n0 = _lib.lp_tv_workspace_bytes_frames_varlen(pk.n, pk.total, M, pf.total, chunk)
    n1 = _lib.lp_tv_workspace_bytes_frames_varlen_cached(pk.n, pk.total, M, pf.total, chunk)
    nscan = _lib.lp_tv_workspace_bytes_varlen(pk.n, pk.total, M, chunk)
    if M == 13:
        assert n1 == n0
    else:
        assert n1 >= n0 + pk.total * M * 4
    got = []
    for nb in (n0, n1):
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
        s = ops.lp_tv_forward_frames_varlen(pk, pf, k, e, zi, chunk=chunk, ws=ws)
        ge, gk, gzi = ops.lp_tv_backward_frames_varlen(pk, pf, gs, k, s, zi, chunk=chunk, ws=ws,
                                                       reuse_forward=True)
        torch.cuda.synchronize()
        assert _lib.lp_tv_device_status() == 0
        got.append([x.cpu().numpy() for x in (s, ge, gk, gzi)])
        if nb == n1 and M == 22:
            base = ((nscan + 255) // 256) * 256
            rows = ws[base:base + pk.total * M * 4].view(torch.float32).reshape(pk.total, M).cpu().numpy()
            for b, n in enumerate(lengths):
                if n == 0:
                    continue
                o = int(pk.offsets[b].item())
                ref = O.coeffs(ks[b][None], n, hop)[0]
                err = np.abs(rows[o:o + n] - ref).max() / max(np.abs(ref).max(), 1e-30)
                assert err <= TOL_F32, (b, err)
    for x, y in zip(*got):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("reuse", [True, False])
def test_frames_resonant_with_and_without_row_cache(reuse):
    """Resonant frames (literal generator, |k| <= 0.8, no per-order decay):
    the defect correction re-runs listed chunks, from generated rows without
    the row cache and from the cached rows with it.  Both give the same bits.
    The filter is checked against the oracle run on the rows the kernels
    generated (kept by the row cache), since on resonant filters the FP32
    rounding of a(t) alone is amplified; dL/dk against the oracle's adjoint
    of the step-up on two signals (it is O(M^3) per sample)."""
    B, T, M, hop = 4, 48000, 22, 120
    rng = np.random.default_rng(61)
    k = inputs.reflection_frames(rng, B, O.n_frames(T, hop), M, 0.8, 1.0).astype(np.float32)
    e = inputs.pulse_train(rng, B, T).astype(np.float32) + 0.1 * rng.standard_normal((B, T)).astype(np.float32)
    gs = rng.standard_normal((B, T)).astype(np.float32)
    kt, et, gst = _t(k), _t(e), _t(gs)
    got = []
    for cache in (False, True):
        ws = ops.workspace_frames(B, T, M, hop, 0, DEV, cache_rows=cache)
        s = ops.lp_tv_forward_frames(kt, et, hop, chunk=0, ws=ws)
        ge, gk, _ = ops.lp_tv_backward_frames(gst, kt, s, hop, need_gzi=False, ws=ws, reuse_forward=reuse)
        torch.cuda.synchronize()
        assert _lib.lp_tv_device_status() == 0
        got.append([x.cpu().numpy() for x in (s, ge, gk)])
        if cache:
            n0 = _lib.lp_tv_workspace_bytes_frames(B, T, M, hop, 0)
            rows = ws[n0:n0 + B * T * M * 4].view(torch.float32).reshape(B, T, M).cpu().numpy()
    for x, y in zip(*got):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    s, ge, gk = got[1]
    rs, rge, rga, _ = O.forward_backward(rows, e, gs)
    _close("s", s, rs)
    _close("ge", ge, rge)
    sel = [0, B - 1]
    _close("gk", gk[sel], O.coeffs_adjoint(k[sel], rga[sel], hop))
