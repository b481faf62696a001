"""Varlen batches: signals of different lengths packed back to back in one
call (lp_tv_forward_varlen_* / lp_tv_backward_varlen_*), against the FP64
oracle signal by signal, and each signal's results alone vs in the mix.

The uneven-batching workload: signal lengths uniform over a range, orders
drawn from {16, 22, 30} (one call per order), stable reflection
coefficients at hop 120 -- here at a size the oracle checks in seconds.
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


def _signals(lengths, M, seed, zi=True, gen="stable", kmax=0.95):
    """One workload per signal (float32 arrays), stable generator by default."""
    ws = [inputs.make("vl", 1, max(n, 1), M, seed=seed + 31 * k, gen=gen, kmax=kmax, with_zi=zi,
                      excitation="pulse" if gen == "literal" else "noise")
          for k, n in enumerate(lengths)]
    return [(w.a[0, :n], w.e[0, :n], w.gs[0, :n], None if w.zi is None else w.zi[0]) for w, n in zip(ws, lengths)]


def _run(sig, M, chunk=0, zi=True, reuse=True):
    lengths = [x[0].shape[0] for x in sig]
    pk = ops.Packed(lengths, DEV)
    a = pk.pack([torch.tensor(x[0], device=DEV) for x in sig], width=M)
    e = pk.pack([torch.tensor(x[1], device=DEV) for x in sig])
    gs = pk.pack([torch.tensor(x[2], device=DEV) for x in sig])
    z = torch.tensor(np.stack([x[3] for x in sig]), device=DEV) if zi else None
    nb = _lib.lp_tv_workspace_bytes_varlen(pk.n, pk.total, M, chunk)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
    s = ops.lp_tv_forward_varlen(pk, a, e, z, chunk=chunk, ws=ws)
    ge, ga, gzi = ops.lp_tv_backward_varlen(pk, gs, a, s, z, need_gzi=zi, chunk=chunk, ws=ws, reuse_forward=reuse)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    out = []
    for k in range(pk.n):
        out.append((pk.unpack(s)[k].cpu().numpy(), pk.unpack(ge)[k].cpu().numpy(), pk.unpack(ga)[k].cpu().numpy(),
                    None if gzi is None else gzi[k].cpu().numpy()))
    return out


def _check_oracle(sig, got, zi=True):
    for (a, e, gs, z), (s, ge, ga, gzi) in zip(sig, got):
        if a.shape[0] == 0:
            continue
        rs, rge, rga, rgzi = O.forward_backward(a[None], e[None], gs[None], z[None] if zi else None)
        for name, x, r in (("s", s, rs), ("ge", ge, rge), ("ga", ga, rga)):
            err = norm_err(x[None], r)
            assert err.max() <= TOL_F32, (name, a.shape[0], err)
        if zi:
            d = np.abs(gzi - rgzi[0]).max() / max(np.abs(rge).max(), 1e-30)
            assert d <= TOL_F32


@pytest.mark.parametrize("M", [16, 22])
@pytest.mark.parametrize("zi", [True, False])
@pytest.mark.parametrize("reuse", [True, False])
def test_varlen_matches_oracle(M, zi, reuse):
    lengths = [5000, 0, 17, 160, 161, 3001, 1, 4800, 999]
    sig = _signals(lengths, M, seed=40 + M, zi=True)
    got = _run(sig, M, zi=zi, reuse=reuse)
    _check_oracle(sig, got, zi=zi)


def test_varlen_alone_equals_in_the_mix():
    """With a fixed chunk length a signal's results do not depend on the
    rest of the batch, bit for bit."""
    M, chunk = 22, 160
    lengths = [4000, 123, 9000, 2048, 777]
    sig = _signals(lengths, M, seed=77)
    mix = _run(sig, M, chunk=chunk)
    for k in range(len(sig)):
        alone = _run([sig[k]], M, chunk=chunk)[0]
        for x, y in zip(alone, mix[k]):
            assert np.array_equal(x, y)


def test_varlen_alone_equals_in_the_mix_resonant():
    """Resonant signals (literal generator, |k| <= 0.8), whose chunks the
    defect correction re-runs: its decisions depend on each signal's own
    values, so results are still the same bits alone and in the mix, and
    within the parity bound of the oracle."""
    M, chunk = 22, 160
    lengths = [48000, 7000, 30001, 160]
    sig = _signals(lengths, M, seed=5, gen="literal", kmax=0.8)
    mix = _run(sig, M, chunk=chunk)
    _check_oracle(sig, mix)
    for k in range(len(sig)):
        alone = _run([sig[k]], M, chunk=chunk)[0]
        for x, y in zip(alone, mix[k]):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("reuse", [True, False])
def test_varlen_chain_lengths_across_warp_splits(reuse):
    """M=22 at chunk 32, signals whose chains have 0, 1, 8, 9, 10, 17, 18,
    27, 35, 36, 37 and 40 group steps in one call: each chain block picks
    the register chain (four warps of up to nine steps) or, past 36 steps,
    the shared-memory chain for its own signal."""
    lengths = [1, 33, 769, 865, 961, 2721, 2881, 6049, 10081, 11521, 11841, 14081]
    sig = _signals(lengths, 22, seed=77)
    _check_oracle(sig, _run(sig, 22, chunk=32, reuse=reuse))


def test_varlen_equals_uniform_call():
    """Equal lengths: the varlen call reproduces the uniform call bit for bit."""
    M, chunk, B, T = 22, 160, 4, 3200
    w = inputs.make("vu", B, T, M, seed=5, gen="stable", with_zi=True)
    sig = [(w.a[b], w.e[b], w.gs[b], w.zi[b]) for b in range(B)]
    got = _run(sig, M, chunk=chunk)
    a, e, gs, zi = (torch.tensor(x, device=DEV) for x in (w.a, w.e, w.gs, w.zi))
    ws = ops.workspace(B, T, M, chunk, torch.float32, DEV)
    s = ops.lp_tv_forward(a, e, zi, chunk=chunk, ws=ws)
    ge, ga, gzi = ops.lp_tv_backward(gs, a, s, zi, chunk=chunk, ws=ws, reuse_forward=True)
    for b in range(B):
        assert np.array_equal(got[b][0], s[b].cpu().numpy())
        assert np.array_equal(got[b][1], ge[b].cpu().numpy())
        assert np.array_equal(got[b][2], ga[b].cpu().numpy())
        assert np.array_equal(got[b][3], gzi[b].cpu().numpy())


def test_uneven_batching_orders_16_22_30():
    """Uneven batch (reduced size): lengths uniform in [1200, 24000], orders
    from {16, 22, 30}, one varlen call per order, each signal against the
    oracle."""
    rng = np.random.default_rng(4)
    n = 24
    lengths = rng.integers(1200, 24001, size=n).tolist()
    orders = rng.choice([16, 22, 30], size=n).tolist()
    for M in (16, 22, 30):
        idx = [k for k in range(n) if orders[k] == M]
        if not idx:
            continue
        sig = _signals([lengths[k] for k in idx], M, seed=900 + M)
        got = _run(sig, M)
        _check_oracle(sig, got)


def test_varlen_checkpoints_match_uniform():
    M, chunk, B, T = 16, 96, 3, 2000
    w = inputs.make("vck", B, T, M, seed=6, gen="stable", with_zi=True)
    pk = ops.Packed([T] * B, DEV)
    a = pk.pack([torch.tensor(w.a[b], device=DEV) for b in range(B)], width=M)
    e = pk.pack([torch.tensor(w.e[b], device=DEV) for b in range(B)])
    zi = torch.tensor(w.zi, device=DEV)
    _, ck = ops.lp_tv_forward_varlen(pk, a, e, zi, chunk=chunk, ckpt=True)
    _, cku = ops.lp_tv_forward(torch.tensor(w.a, device=DEV), torch.tensor(w.e, device=DEV), zi, chunk=chunk,
                               ckpt=True)
    assert torch.equal(ck, cku.reshape(-1, M))


def test_uneven_full_length_sampled():
    """Full lengths of the uneven workload (up to 240000 samples) at the
    largest order, 30: inputs drawn on the GPU with the same recipe; the
    longest and two other signals are checked against the oracle in full."""
    M = 30
    lengths = [240000, 12000, 150001, 99999, 200000, 12345]
    sig_t = inputs.signals_torch(lengths, M, seed=55, gen="stable", device=DEV)
    pk = ops.Packed(lengths, DEV)
    a = pk.pack([x[0] for x in sig_t], width=M)
    e = pk.pack([x[1] for x in sig_t])
    gs = pk.pack([x[2] for x in sig_t])
    s = ops.lp_tv_forward_varlen(pk, a, e)
    ge, ga, _ = ops.lp_tv_backward_varlen(pk, gs, a, s, need_gzi=False)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    for k in (0, 2, 5):
        an, en, gn = (x.cpu().numpy() for x in sig_t[k])
        rs, rge, rga, _ = O.forward_backward(an[None], en[None], gn[None])
        for name, x, r in (("s", pk.unpack(s)[k], rs), ("ge", pk.unpack(ge)[k], rge), ("ga", pk.unpack(ga)[k], rga)):
            err = norm_err(x.cpu().numpy()[None], r)
            assert err.max() <= TOL_F32, (name, k, err)


# ---------------------------------------------------------------------------
# Mixed orders in one call (lp_tv_*_mixed_f32)
# ---------------------------------------------------------------------------
def _mixed_signals(lengths, orders, seed, gen="stable", kmax=0.95, zi=True):
    out = []
    for k, (n, m) in enumerate(zip(lengths, orders)):
        w = inputs.make("mx", 1, max(n, 1), m, seed=seed + 31 * k, gen=gen, kmax=kmax, with_zi=zi,
                        excitation="pulse" if gen == "literal" else "noise")
        out.append((w.a[0, :n], w.e[0, :n], w.gs[0, :n], None if w.zi is None else w.zi[0]))
    return out


def _run_mixed(sig, orders, chunk=0, zi=True, reuse=True):
    lengths = [x[0].shape[0] for x in sig]
    pm = ops.PackedMixed(lengths, orders, DEV)
    a = pm.pack_coeffs([torch.tensor(x[0], device=DEV) for x in sig])
    e = pm.pack_rows([torch.tensor(x[1], device=DEV) for x in sig])
    gs = pm.pack_rows([torch.tensor(x[2], device=DEV) for x in sig])
    z = None
    if zi:
        z = torch.zeros((pm.n, 32), device=DEV)
        for b, x in enumerate(sig):
            z[b, :orders[b]] = torch.tensor(x[3], device=DEV)
    ws = pm.workspace(chunk)
    s = ops.lp_tv_forward_mixed(pm, a, e, z, chunk=chunk, ws=ws)
    ge, ga, gzi = ops.lp_tv_backward_mixed(pm, gs, a, s, z, need_gzi=zi, chunk=chunk, ws=ws, reuse_forward=reuse)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    out = []
    for b in range(pm.n):
        out.append((pm.unpack_rows(s)[b].cpu().numpy(), pm.unpack_rows(ge)[b].cpu().numpy(),
                    pm.unpack_coeffs(ga)[b].cpu().numpy(),
                    None if gzi is None else gzi[b, :orders[b]].cpu().numpy()))
    return out


@pytest.mark.parametrize("reuse", [True, False])
@pytest.mark.parametrize("zi", [True, False])
def test_mixed_orders_match_oracle(reuse, zi):
    """Signals of orders 16, 22, 30 and of orders that pad (5, 17, 26) with
    ragged and empty lengths, in one call per direction."""
    lengths = [5000, 0, 3001, 160, 161, 2400, 1, 4800, 999, 777, 1500]
    orders = [16, 22, 30, 22, 16, 30, 5, 17, 26, 30, 22]
    sig = _mixed_signals(lengths, orders, seed=300)
    got = _run_mixed(sig, orders, zi=zi, reuse=reuse)
    _check_oracle(sig, got, zi=zi)


def test_mixed_orders_alone_equals_in_the_mix_and_single_order_calls():
    """With a fixed chunk: every signal's results are the same bits alone,
    in the mixed batch, and in a single-order varlen call of its order."""
    chunk = 160
    lengths = [4000, 123, 9000, 2048, 777, 3500]
    orders = [16, 30, 22, 16, 22, 30]
    sig = _mixed_signals(lengths, orders, seed=700)
    mix = _run_mixed(sig, orders, chunk=chunk)
    for k in range(len(sig)):
        alone = _run_mixed([sig[k]], [orders[k]], chunk=chunk)[0]
        single = _run([sig[k]], orders[k], chunk=chunk)[0]
        for x, y, z in zip(alone, mix[k], single):
            assert np.array_equal(x, y)
            assert np.array_equal(x, z)


def test_mixed_resonant_signals():
    """Resonant signals (literal generator, |k| <= 0.8) of three orders in
    one call: the defect correction runs per order group.  (At order 30
    this generator diverges, max |s| about 1e25: beyond FP32 for any
    algorithm, so the orders here stop at 22.)"""
    lengths = [48000, 30000, 20000, 48000]
    orders = [22, 16, 12, 22]
    sig = _mixed_signals(lengths, orders, seed=5, gen="literal", kmax=0.8, zi=False)
    got = _run_mixed(sig, orders, zi=False)
    _check_oracle(sig, got, zi=False)


def test_uneven_batching_one_call():
    """The uneven workload (reduced size): lengths uniform in [1200, 24000],
    orders drawn from {16, 22, 30}, all in one mixed call per direction,
    each signal against the oracle."""
    rng = np.random.default_rng(4)
    n = 24
    lengths = rng.integers(1200, 24001, size=n).tolist()
    orders = rng.choice([16, 22, 30], size=n).tolist()
    sig = _mixed_signals(lengths, orders, seed=900)
    got = _run_mixed(sig, orders)
    _check_oracle(sig, got)


def test_mixed_invalid_orders():
    pm_ok = ops.PackedMixed([10, 20], [4, 8], DEV)
    with pytest.raises(ValueError):
        ops.PackedMixed([10, 20], [4, 40], DEV).workspace()
    assert pm_ok.total_a == 40 + 160
