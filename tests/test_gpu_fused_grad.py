"""Eq. 12 inside the adjoint re-run.

With LP_BWD_FUSED_GA and M one of the compiled orders, the chunked adjoint
re-run writes ga(t) = -ge(t) s(t-i) as it produces ge(t), and the rows leave
shared memory by bulk stores (plain stores for a ragged last stage or rows
that are not 16-byte aligned).  Without it a separate pass over ge and s
writes ga.  Both compute each element as the same single product, so they
must agree bit for bit, and the fused one must match the FP64 oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2406_05128_gb300 import _lib, inputs, ops  # noqa: E402
from tests.helpers import TOL_F32, TOL_F64, assert_close  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


def _uniform(w, dtype, chunk, reuse, zi):
    a = torch.tensor(w.a, dtype=dtype, device=DEV)
    e = torch.tensor(w.e, dtype=dtype, device=DEV)
    gs = torch.tensor(w.gs, dtype=dtype, device=DEV)
    z = torch.tensor(w.zi, dtype=dtype, device=DEV) if zi else None
    B, T, M = a.shape
    ws = ops.workspace(B, T, M, chunk, dtype, DEV)
    s = ops.lp_tv_forward(a, e, z, chunk=chunk, ws=ws)
    out = []
    for fused in (True, False):
        ge, ga, gzi = ops.lp_tv_backward(gs, a, s, z, chunk=chunk, ws=ws, reuse_forward=reuse, fused_ga=fused)
        torch.cuda.synchronize()
        assert _lib.lp_tv_device_status() == 0
        out.append((ge.cpu().numpy(), ga.cpu().numpy(), None if gzi is None else gzi.cpu().numpy()))
    return s.cpu().numpy(), out


def _same_bits(x, y):
    if x is None or y is None:
        assert x is None and y is None
        return
    assert np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("B,T,M,chunk,reuse,zi", [
    (2, 1237, 16, 0, True, True),     # ragged last stage and chunk
    (3, 1000, 22, 48, True, True),    # many chunks, each stage full
    (2, 3001, 22, 0, False, True),    # adjoint with its own transfers
    (2, 7, 22, 0, True, True),        # T < M: every row reaches into zi
    (2, 1500, 30, 0, True, False),
    (2, 999, 32, 0, True, True),
    (3, 640, 4, 32, True, True),
    (2, 800, 5, 0, True, True),       # padded order: the separate pass either way
])
def test_fused_equals_separate_and_oracle_f32(B, T, M, chunk, reuse, zi):
    w = inputs.make("fg", B, T, M, seed=900 + T + M, gen="stable", with_zi=True)
    _, ((ge, ga, gzi), (ge2, ga2, gzi2)) = _uniform(w, torch.float32, chunk, reuse, zi)
    _same_bits(ge, ge2)
    _same_bits(ga, ga2)
    _same_bits(gzi, gzi2)
    rs, rge, rga, rgzi = O.forward_backward(w.a, w.e, w.gs, w.zi if zi else None)
    assert_close("ga", ga, rga, TOL_F32)


@pytest.mark.parametrize("M", [8, 12])
def test_fused_equals_separate_and_oracle_f64(M):
    w = inputs.make("fg64", 2, 1111, M, seed=77 + M, gen="stable", with_zi=True)
    _, ((ge, ga, gzi), (ge2, ga2, gzi2)) = _uniform(w, torch.float64, 0, True, True)
    _same_bits(ga, ga2)
    _same_bits(ge, ge2)
    rs, rge, rga, rgzi = O.forward_backward(w.a, w.e, w.gs, w.zi)
    assert_close("ga", ga, rga, TOL_F64)


def test_varlen_odd_offsets_fused():
    """Odd offsets put rows off the 16-byte grid (plain stores), with an
    empty signal and lengths that end mid-stage."""
    M = 22
    lengths = [101, 0, 999, 33, 1600, 7]
    sig = [inputs.make("fv", 1, max(n, 1), M, seed=40 + k, gen="stable", with_zi=True) for k, n in enumerate(lengths)]
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    total = int(off[-1])
    a = torch.tensor(np.concatenate([w.a[0, :n] for w, n in zip(sig, lengths)]), device=DEV).contiguous()
    e = torch.tensor(np.concatenate([w.e[0, :n] for w, n in zip(sig, lengths)]), device=DEV)
    gs = torch.tensor(np.concatenate([w.gs[0, :n] for w, n in zip(sig, lengths)]), device=DEV)
    zi = torch.tensor(np.stack([w.zi[0] for w in sig]), device=DEV)
    offs = torch.tensor(off, device=DEV)
    n = len(lengths)
    code = _lib.LP_DTYPE_F32
    nb = _lib.lp_tv_workspace_bytes_varlen(n, total, M, 0, code)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
    st = torch.cuda.current_stream().cuda_stream
    s = torch.empty(total, device=DEV)
    _lib.lp_tv_forward_varlen(code, n, offs.data_ptr(), total, M, a.data_ptr(), e.data_ptr(), zi.data_ptr(),
                              s.data_ptr(), None, 0, ws.data_ptr(), ws.numel(), st)
    res = []
    for flags in (_lib.LP_BWD_REUSE_FORWARD | _lib.LP_BWD_FUSED_GA, _lib.LP_BWD_REUSE_FORWARD):
        ge = torch.empty(total, device=DEV)
        ga = torch.full((total, M), float("nan"), device=DEV)
        gzi = torch.empty((n, M), device=DEV)
        _lib.lp_tv_backward_varlen(code, n, offs.data_ptr(), total, M, gs.data_ptr(), a.data_ptr(), s.data_ptr(),
                                   zi.data_ptr(), ge.data_ptr(), ga.data_ptr(), gzi.data_ptr(), 0, flags,
                                   ws.data_ptr(), ws.numel(), st)
        torch.cuda.synchronize()
        assert _lib.lp_tv_device_status() == 0
        res.append((ge.cpu().numpy(), ga.cpu().numpy(), gzi.cpu().numpy()))
    (ge, ga, gzi), (ge2, ga2, gzi2) = res
    _same_bits(ge, ge2)
    _same_bits(ga, ga2)
    _same_bits(gzi, gzi2)
    for k, (w, L) in enumerate(zip(sig, lengths)):
        if L == 0:
            continue
        rs, rge, rga, rgzi = O.forward_backward(w.a[:, :L], w.e[:, :L], w.gs[:, :L], w.zi)
        assert_close(f"ga[{k}]", ga[off[k]:off[k + 1]][None], rga, TOL_F32)


def test_recompute_fused_equals_separate():
    B, T, M, chunk = 2, 2000, 22, 80
    w = inputs.make("fr", B, T, M, seed=5, gen="stable", with_zi=True)
    a = torch.tensor(w.a, device=DEV)
    e = torch.tensor(w.e, device=DEV)
    gs = torch.tensor(w.gs, device=DEV)
    z = torch.tensor(w.zi, device=DEV)
    ws = ops.workspace(B, T, M, chunk, torch.float32, DEV)
    _, ckpt = ops.lp_tv_forward(a, e, z, chunk=chunk, ws=ws, ckpt=True)
    got = []
    for fused in (True, False):
        ge, ga, gzi = ops.lp_tv_backward_recompute(gs, a, e, ckpt, z, chunk=chunk, ws=ws, reuse_forward=True,
                                                   fused_ga=fused)
        torch.cuda.synchronize()
        got.append([x.cpu().numpy() for x in (ge, ga, gzi)])
    for x, y in zip(*got):
        _same_bits(x, y)


def test_headline_size_fused_equals_separate():
    """B=32, T=48000, M=22 as the bench runs it (chunk 160, reused
    transfers): the fused rows equal the separate pass everywhere."""
    B, T, M = 32, 48000, 22
    w = inputs.batched_headline(seed=2, gen="literal", B=B, T=T, M=M)
    _, ((ge, ga, _), (ge2, ga2, _)) = _uniform(w, torch.float32, 160, True, False)
    _same_bits(ge, ge2)
    _same_bits(ga, ga2)


@pytest.mark.parametrize("reuse,zi", [(True, True), (False, False)])
def test_resonant_fused_equals_separate(reuse, zi):
    """Resonant signals (literal generator, |k| <= 0.8): the defect
    correction re-runs listed chunks of the adjoint, and in the fused path
    that second pass writes their ga rows again.  Both paths take the same
    steps, so ge, ga and gzi agree bit for bit, and meet the oracle."""
    w = inputs.make("resfg", 4, 48000, 22, seed=5, kmax=0.8, gen="literal", excitation="pulse", with_zi=zi)
    s, ((ge, ga, gzi), (ge2, ga2, gzi2)) = _uniform(w, torch.float32, 0, reuse, zi)
    _same_bits(ge, ge2)
    _same_bits(ga, ga2)
    _same_bits(gzi, gzi2)
    rs, rge, rga, _ = O.forward_backward(w.a, w.e, w.gs, w.zi if zi else None)
    assert_close("s", s, rs, TOL_F32)
    assert_close("ge", ge, rge, TOL_F32)
    assert_close("ga", ga, rga, TOL_F32)
