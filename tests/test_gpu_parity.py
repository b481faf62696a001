"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: per signal, max |gpu - oracle| / max |oracle| <= 1e-4 for FP32
outputs (s, dL/de, dL/da, dL/dzi) on stable coefficients, <= 1e-10 for FP64.
Inputs are the same float32 (or float64) arrays on both sides.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2406_05128_gb300 import _lib, inputs, ops  # noqa: E402
from tests.helpers import TOL_F32, TOL_F64, assert_close, norm_err  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


def _run(w, dtype=torch.float32, chunk=0, algo="chunked", zi=True, reuse=True):
    """Forward then adjoint through the C ABI.  With reuse (the default for
    the chunked algorithm) the adjoint reuses the forward's chunk transfers
    from the shared workspace; otherwise it computes its own."""
    a = torch.tensor(w.a, dtype=dtype, device=DEV)
    e = torch.tensor(w.e, dtype=dtype, device=DEV)
    gs = torch.tensor(w.gs, dtype=dtype, device=DEV)
    z = torch.tensor(w.zi, dtype=dtype, device=DEV) if (zi and w.zi is not None) else None
    B, T, M = a.shape
    ws = ops.workspace(B, T, M, chunk, dtype, DEV)
    s = ops.lp_tv_forward(a, e, z, chunk=chunk, algo=algo, ws=ws)
    reuse = reuse and algo == "chunked"
    ge, ga, gzi = ops.lp_tv_backward(gs, a, s, z, chunk=chunk, algo=algo, need_gzi=True, ws=ws,
                                     reuse_forward=reuse)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    return [x.cpu().numpy() for x in (s, ge, ga, gzi)]


def _oracle(w, zi=True):
    z = w.zi if zi else None
    return O.forward_backward(w.a, w.e, w.gs, z)


def _compare(w, got, tol, zi=True):
    s, ge, ga, gzi = got
    rs, rge, rga, rgzi = _oracle(w, zi)
    out = {"s": assert_close("s", s, rs, tol),
           "ge": assert_close("ge", ge, rge, tol),
           "ga": assert_close("ga", ga, rga, tol)}
    if zi and w.zi is not None:
        # the initial-state gradient is a short sum; normalise by the scale of ge
        d = np.abs(gzi - rgzi).max(axis=1) / np.abs(rge).max(axis=1)
        assert d.max() <= tol, f"gzi: {d.max():.3e}"
    return out


CASES = [
    # B, T, M, chunk, zi
    (1, 1, 1, 0, False),
    (2, 5, 3, 0, True),
    (3, 7, 12, 0, True),       # T < M
    (2, 500, 1, 0, True),
    (2, 1000, 4, 64, True),
    (3, 1237, 16, 0, True),    # ragged tail
    (2, 2000, 22, 44, True),   # many short chunks
    (2, 3001, 22, 0, True),
    (2, 1500, 30, 0, True),
    (2, 999, 32, 0, True),
    (4, 777, 5, 0, True),      # padded order (5 -> 8)
    (2, 640, 13, 32, True),    # padded order (13 -> 16), chunk rounded up
    (5, 4096, 22, 22, False),  # chunk = one stage
    (1, 48000, 22, 0, True),
]


@pytest.mark.parametrize("B,T,M,chunk,zi", CASES)
@pytest.mark.parametrize("algo", ["chunked", "chunked-own-adjoint", "plain"])
def test_parity_f32(B, T, M, chunk, zi, algo):
    if algo == "plain" and T > 5000:
        pytest.skip("plain path covered at smaller T")
    w = inputs.make("case", B, T, M, seed=B * 1000 + T + M, gen="stable", with_zi=zi)
    own = algo == "chunked-own-adjoint"
    _compare(w, _run(w, chunk=chunk, algo="chunked" if own else algo, zi=zi, reuse=not own), TOL_F32, zi)


@pytest.mark.parametrize("B,T,M,chunk", [(2, 300, 4, 0), (3, 1001, 16, 48), (2, 77, 9, 0), (1, 5, 2, 0)])
@pytest.mark.parametrize("algo", ["chunked", "chunked-own-adjoint", "plain"])
def test_parity_f64(B, T, M, chunk, algo):
    w = inputs.make("case64", B, T, M, seed=77 + T, gen="stable", with_zi=True)
    w.a, w.e, w.gs, w.zi = (x.astype(np.float64) for x in (w.a, w.e, w.gs, w.zi))
    own = algo == "chunked-own-adjoint"
    _compare(w, _run(w, dtype=torch.float64, chunk=chunk, algo="chunked" if own else algo, reuse=not own), TOL_F64)


def test_plain_small_config():
    """B=1, T=4800, M=16, k ~ U(-0.9, 0.9) without decay (the literal small workload)."""
    w = inputs.plain_small(seed=1, gen="literal")
    errs = _compare(w, _run(w, zi=False), TOL_F32, zi=False)
    print("plain small config errors", errs)


def test_headline_config_stable_full_size():
    """B=32, T=48000, M=22 at the benchmark's launch configuration (auto
    chunk), every sample of every signal against the oracle."""
    w = inputs.batched_headline(seed=2, gen="stable")
    errs = _compare(w, _run(w, zi=False), TOL_F32, zi=False)
    print("headline config (stable) errors", errs)


_LIT08 = {}


def _lit08(B):
    """The literal uniform generator at |k| <= 0.8 (no per-order decay),
    pulse-train excitation, T=48000, M=22, and its oracle results."""
    if B not in _LIT08:
        w = inputs.make("lit08", B, 48000, 22, seed=5, kmax=0.8, gen="literal", excitation="pulse")
        _LIT08[B] = (w, _oracle(w, zi=False))
    return _LIT08[B]


@pytest.mark.parametrize("B", [8, 32])
@pytest.mark.parametrize("pick", ["default", "tuned"])
@pytest.mark.parametrize("reuse", [True, False])
def test_literal_generator_k08_ill_conditioned(B, pick, reuse):
    """Some signals of the literal generator at |k| <= 0.8 are resonant and
    ill-conditioned: in FP32 the chunk transfers' rounding, amplified along
    the chain of chunk states, reached 2e-4 (B=8) and about 6e-4 (B=32)
    before the defect correction.  With it the chunked scan meets the 1e-4
    bound like the plain sequential recursion, at the library's default
    chunk and at the autotuner's pick, with reused and with its own adjoint
    transfers."""
    from paper_2406_05128_gb300 import autotune
    w, ref = _lit08(B)
    chunk = 0 if pick == "default" else autotune.tune_uniform(B, 48000, 22)[0]
    got = _run(w, zi=False, chunk=chunk, reuse=reuse)
    for name, i in (("s", 0), ("ge", 1), ("ga", 2)):
        ec = norm_err(got[i], ref[i])
        print(f"literal k<=0.8 B={B} chunk={chunk} reuse={reuse} {name}: max {ec.max():.2e}")
        assert np.all(ec <= TOL_F32), (name, ec)


def test_literal_generator_k08_plain_and_fused():
    """The same workload through the plain sequential kernel, and through
    the chunked adjoint that writes ga in its re-run (LP_BWD_FUSED_GA)."""
    w, ref = _lit08(8)
    got_p = _run(w, zi=False, algo="plain")
    a = torch.tensor(w.a, device=DEV)
    e = torch.tensor(w.e, device=DEV)
    gs = torch.tensor(w.gs, device=DEV)
    B, T, M = a.shape
    ws = ops.workspace(B, T, M, 0, torch.float32, DEV)
    s = ops.lp_tv_forward(a, e, ws=ws)
    ge, ga, _ = ops.lp_tv_backward(gs, a, s, ws=ws, reuse_forward=True, fused_ga=True, need_gzi=False)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    got_f = [x.cpu().numpy() for x in (s, ge, ga)]
    for name, i in (("s", 0), ("ge", 1), ("ga", 2)):
        assert np.all(norm_err(got_p[i], ref[i]) <= TOL_F32), name
        assert np.all(norm_err(got_f[i], ref[i]) <= TOL_F32), name


def test_zero_coefficients_identity():
    B, T, M = 3, 1000, 22
    a = torch.zeros((B, T, M), device=DEV)
    e = torch.randn((B, T), device=DEV)
    gs = torch.randn((B, T), device=DEV)
    s = ops.lp_tv_forward(a, e)
    ge, ga, _ = ops.lp_tv_backward(gs, a, s)
    assert torch.equal(s, e) and torch.equal(ge, gs)
    e_np, gs_np = e.cpu().numpy(), gs.cpu().numpy()
    want = np.zeros((B, T, M), np.float32)
    for i in range(1, M + 1):
        want[:, i:, i - 1] = -gs_np[:, i:] * e_np[:, :-i]
    assert np.array_equal(ga.cpu().numpy(), want)


def test_deterministic_and_chunk_invariant():
    w = inputs.make("det", 4, 20000, 22, seed=9, gen="stable", with_zi=True)
    r1 = _run(w)
    r2 = _run(w)
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)
    r3 = _run(w, chunk=132)
    for x, y in zip(r1[:3], r3[:3]):
        assert norm_err(x, y).max() < 1e-5


def test_degenerate_sizes():
    a = torch.zeros((0, 10, 4), device=DEV)
    e = torch.zeros((0, 10), device=DEV)
    assert ops.lp_tv_forward(a, e).shape == (0, 10)
    a = torch.zeros((2, 0, 4), device=DEV)
    e = torch.zeros((2, 0), device=DEV)
    s = ops.lp_tv_forward(a, e)
    ge, ga, gzi = ops.lp_tv_backward(e, a, s, torch.zeros((2, 4), device=DEV))
    assert s.shape == (2, 0) and gzi.shape == (2, 4) and torch.all(gzi == 0)
    # M = 0: the filter is the identity
    a = torch.zeros((2, 50, 0), device=DEV)
    e = torch.randn((2, 50), device=DEV)
    s = ops.lp_tv_forward(a, e)
    ge, ga, gzi = ops.lp_tv_backward(e, a, s)
    assert torch.equal(s, e) and torch.equal(ge, e)


def test_invalid_arguments_raise():
    a = torch.zeros((2, 10, 40), device=DEV)
    e = torch.zeros((2, 10), device=DEV)
    with pytest.raises(_lib.LPError):
        ops.lp_tv_forward(a, e)  # order 40 is not supported
    a = torch.zeros((2, 10, 4), device=DEV)
    ws = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(_lib.LPError):
        ops.lp_tv_forward(a, e, ws=ws)  # workspace too small
    with pytest.raises(ValueError):
        ops.lp_tv_forward(a.cpu(), e.cpu())  # no CPU path


def test_gradcheck_f64():
    """torch.autograd.gradcheck in FP64 at B=2, T=256, M=4 through the
    differentiable op (chunked scan with several chunks)."""
    torch.manual_seed(0)
    w = inputs.make("gc", 2, 256, 4, seed=3, gen="stable", with_zi=True)
    a = torch.tensor(w.a, dtype=torch.float64, device=DEV, requires_grad=True)
    e = torch.tensor(w.e, dtype=torch.float64, device=DEV, requires_grad=True)
    zi = torch.tensor(w.zi, dtype=torch.float64, device=DEV, requires_grad=True)
    fn = lambda a_, e_, z_: ops.lp_filter(a_, e_, z_, chunk=32)
    assert torch.autograd.gradcheck(fn, (a, e, zi), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_autograd_matches_oracle_f32():
    w = inputs.make("ag", 3, 5000, 22, seed=11, gen="stable", with_zi=True)
    a = torch.tensor(w.a, device=DEV, requires_grad=True)
    e = torch.tensor(w.e, device=DEV, requires_grad=True)
    zi = torch.tensor(w.zi, device=DEV, requires_grad=True)
    s = ops.lp_filter(a, e, zi)
    s.backward(torch.tensor(w.gs, device=DEV))
    rs, rge, rga, rgzi = _oracle(w)
    assert_close("s", s.detach().cpu().numpy(), rs, TOL_F32)
    assert_close("ge", e.grad.cpu().numpy(), rge, TOL_F32)
    assert_close("ga", a.grad.cpu().numpy(), rga, TOL_F32)


@pytest.mark.parametrize("shape", [(2, 16), (1, 8), (2, 8)])
def test_parity_launch_shapes(shape):
    """The autotuner's alternative launch shapes (summary lanes per chunk,
    re-run chunks per warp) against the oracle, uniform and varlen."""
    from paper_2406_05128_gb300 import autotune
    w = inputs.make("shape", 3, 7001, 22, seed=41, gen="stable", with_zi=True)
    with autotune.use_shape(shape):
        got = _run(w, chunk=96)
    _compare(w, got, TOL_F32)
    w16 = inputs.make("shape16", 2, 3001, 16, seed=42, gen="stable", with_zi=True)
    with autotune.use_shape(shape):
        got16 = _run(w16, chunk=0, reuse=False)
    _compare(w16, got16, TOL_F32)


def test_autotuner_picks_a_shape():
    from paper_2406_05128_gb300 import autotune
    L, shape, res, res_sh = autotune.tune_uniform(4, 12000, 22, iters=2, shapes=True)
    assert L in res and shape in autotune.SHAPES and set(res_sh) == set(autotune.SHAPES)


def test_scan_without_room_for_chain_blocks():
    """B=40 x 48000 at chunk 160 has 1360 scan items: their 340 blocks fill
    the cooperative grid, so the warp of each signal's first group runs the
    signal's chain (no chain blocks)."""
    w = inputs.make("nochain", 40, 48000, 22, seed=71, gen="stable", with_zi=True)
    _compare(w, _run(w, chunk=160), TOL_F32)


@pytest.mark.parametrize("T", [865, 961, 11521, 11841])
@pytest.mark.parametrize("reuse", [True, False])
def test_scan_chain_split_across_warps(T, reuse):
    """Chains of 9, 10, 36 and 37 group steps at M=22, chunk 32: a chain
    block's four warps take up to nine steps each with their maps in
    registers and hand the state on, so these lengths end a chain at a
    warp's last step, one past it, at the last warp's last step, and one
    step too long for the registers (the shared-memory chain)."""
    w = inputs.make("split", 3, T, 22, seed=73, gen="stable", with_zi=True)
    _compare(w, _run(w, chunk=32, reuse=reuse), TOL_F32)


@pytest.mark.parametrize("M", [17, 21])
def test_scan_chain_split_padded_order(M):
    """Orders padded to 22 take the register chain too: the initial state
    has M < 22 components (chains of 35 steps at chunk 32)."""
    w = inputs.make("splitpad", 3, 10081, M, seed=74 + M, gen="stable", with_zi=True)
    _compare(w, _run(w, chunk=32), TOL_F32)


@pytest.mark.parametrize("reuse", [True, False])
def test_scan_chain_longer_than_chain_ring(reuse):
    """Two signals of 240000 samples at chunk 32: 7500 chunks in groups of
    44, so each chain has 170 group maps, more than a chain block holds at
    once; the chain streams through the halves of its ring (and the item
    warps through theirs, their groups being longer than a warp's ring)."""
    w = inputs.make("longchain", 2, 240000, 22, seed=72, gen="stable", with_zi=True)
    _compare(w, _run(w, chunk=32, reuse=reuse), TOL_F32)
