"""The serving loop on the GPU (include/tvlp_serve.h): continuous batching of
synthesis (forward) and adaptation (forward + adjoint) requests.

- Each request's results are bit for bit the same alone and in a mix where
  requests arrive while others are on the GPU (fixed chunk length; blocks
  that depend only on the request's own length).
- Results match the FP64 oracle on the whole signal within the FP32 parity
  bound, including utterances served in many blocks whose filter state is
  carried on the device from block to block.
- The mix really was batched and overlapped, and stayed within the memory
  budget; a budget that holds about one iteration still serves everything.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2406_05128_gb300 import _lib, inputs, serve  # noqa: E402
from tests.helpers import TOL_F32, norm_err  # noqa: E402

M = 22


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


def _requests(lengths, kinds, seed):
    out = []
    for k, (T, kind) in enumerate(zip(lengths, kinds)):
        w = inputs.make("srv", 1, max(T, 1), M, seed=seed + 17 * k, gen="stable")
        a = torch.from_numpy(np.ascontiguousarray(w.a[0, :T])).pin_memory()
        e = torch.from_numpy(np.ascontiguousarray(w.e[0, :T])).pin_memory()
        gs = torch.from_numpy(np.ascontiguousarray(w.gs[0, :T])).pin_memory() if kind else None
        out.append((a, e, gs))
    return out


def _outputs(req):
    if req.kind == serve.ADAPT:
        return [req.s.numpy().copy(), req.ge.numpy().copy(), req.ga.numpy().copy()]
    return [req.s.numpy().copy()]


CFG = dict(chunk=160, block_rows=4096, max_signals=8, max_iter_rows=1 << 17, max_inflight=3, hbm_budget=256 << 20)
LENGTHS = [4096, 0, 1, 17, 4097, 12000, 30001, 8192, 999, 20000, 2, 16385, 7000, 3000, 45000, 123, 9000, 5000]
KINDS = [0, 0, 0, 1, 0, 1, 0, 0, 1, 0, 0, 0, 1, 0, 0, 1, 0, 0]


def _mix(srv, reqs, rng):
    subs = []
    for a, e, gs in reqs:
        subs.append(srv.submit(a, e, gs))
        time.sleep(float(rng.uniform(0, 3e-4)))
    done = srv.drain(timeout_s=60)
    assert {r.id for r in done} == {r.id for r in subs}
    assert all(r.status == 0 for r in subs)
    return subs


def test_alone_equals_in_the_mix_and_oracle():
    reqs = _requests(LENGTHS, KINDS, seed=300)
    rng = np.random.default_rng(1)
    with serve.Server(M, **CFG) as srv:
        mix = _mix(srv, reqs, rng)
        st = srv.stats()
        alone = []
        for a, e, gs in reqs:
            r = srv.submit(a, e, gs)
            srv.drain(timeout_s=60)
            alone.append(r)
        assert _lib.lp_tv_device_status() == 0
    # the mix was batched, overlapped, carried states, and kept to the budget
    assert st["completed"] == len(reqs) and st["error"] == 0
    assert st["max_signals_iter"] > 1
    assert st["overlapped"] > 0
    assert st["carried_blocks"] > 0
    assert 0 < st["ring_peak"] <= st["ring_bytes"] and st["device_bytes"] <= CFG["hbm_budget"]
    for r_mix, r_alone in zip(mix, alone):
        for x, y in zip(_outputs(r_mix), _outputs(r_alone)):
            assert np.array_equal(x, y), (r_mix.T, r_mix.kind)
    for (a, e, gs), r in zip(reqs, mix):
        if r.T == 0:
            continue
        an, en = a.numpy()[None], e.numpy()[None]
        if r.kind == serve.ADAPT:
            rs, rge, rga, _ = O.forward_backward(an, en, gs.numpy()[None])
            for name, x, ref in (("s", r.s, rs), ("ge", r.ge, rge), ("ga", r.ga, rga)):
                err = norm_err(x.numpy()[None], ref)
                assert err.max() <= TOL_F32, (name, r.T, err)
        else:
            rs = O.forward(an, en)
            err = norm_err(r.s.numpy()[None], rs)
            assert err.max() <= TOL_F32, ("s", r.T, err)


def test_long_utterance_state_carried_across_many_blocks():
    """A 20 s utterance (480000 samples) in blocks of 4096: 118 carried
    filter states, against the oracle on the whole signal."""
    T = 480000
    sig = inputs.signals_torch([T], M, seed=91, gen="stable", device="cuda")[0]
    a, e = (x.cpu().contiguous().pin_memory() for x in sig[:2])
    with serve.Server(M, **CFG) as srv:
        r = srv.submit(a, e)
        srv.drain(timeout_s=60)
        st = srv.stats()
    assert r.status == 0 and st["carried_blocks"] == -(-T // 4096) - 1
    rs = O.forward(a.numpy()[None], e.numpy()[None])
    assert norm_err(r.s.numpy()[None], rs).max() <= TOL_F32


def test_small_budget_serves_everything():
    """A budget whose ring holds about one largest iteration: requests wait
    for memory; results are still those of the roomy server."""
    reqs = _requests(LENGTHS, KINDS, seed=300)
    cfg = dict(CFG, max_iter_rows=1 << 15)
    probe = serve.Server(M, **dict(cfg, hbm_budget=256 << 20))
    fixed = probe.stats()["device_bytes"] - probe.stats()["ring_bytes"]
    probe.close()
    # the ring: one largest region (every row in the adaptation call)
    region = (1 << 15) * (8 * M + 16) + 8192
    with serve.Server(M, **dict(cfg, hbm_budget=fixed + region + 4096)) as srv:
        got = _mix(srv, reqs, np.random.default_rng(2))
        st = srv.stats()
    assert st["ring_peak"] <= st["ring_bytes"] < 2 * region
    with serve.Server(M, **cfg) as srv:
        ref = _mix(srv, reqs, np.random.default_rng(3))
    for x, y in zip(got, ref):
        for u, v in zip(_outputs(x), _outputs(y)):
            assert np.array_equal(u, v)


def test_whole_requests_mode_matches_varlen_call():
    """block_rows=0 serves every request whole: the same numbers as one
    varlen forward call at the same chunk length."""
    from paper_2406_05128_gb300 import ops
    lengths = [5000, 17, 12001, 3000]
    reqs = _requests(lengths, [0] * 4, seed=500)
    with serve.Server(M, **dict(CFG, block_rows=0, max_iter_rows=1 << 16)) as srv:
        got = _mix(srv, reqs, np.random.default_rng(4))
    pk = ops.Packed(lengths, "cuda")
    a = pk.pack([x[0].cuda() for x in reqs], width=M)
    e = pk.pack([x[1].cuda() for x in reqs])
    s = ops.lp_tv_forward_varlen(pk, a, e, chunk=160)
    for r, ref in zip(got, pk.unpack(s)):
        assert np.array_equal(r.s.numpy(), ref.cpu().numpy())


def test_rejects_what_no_iteration_holds():
    with serve.Server(M, **dict(CFG, max_iter_rows=1 << 12)) as srv:
        T = 5000
        a = torch.zeros((T, M)).pin_memory()
        e = torch.zeros(T).pin_memory()
        with pytest.raises(_lib.LPError) as ei:
            srv.submit(a, e, e)  # adaptation runs whole: 5000 rows > 4096
        assert ei.value.code == _lib.LP_ETOOBIG
        r = srv.submit(a, e)  # synthesis is cut into blocks
        srv.drain(timeout_s=30)
        assert r.status == 0 and torch.equal(r.s, e)
        with pytest.raises(ValueError):
            srv.submit(torch.zeros((T, M)), torch.zeros(T))  # not page-locked


def test_frames_server_alone_equals_mix_and_oracle():
    """hop > 0: requests carry reflection coefficients per frame and the
    kernels generate a(t); adaptation requests get dL/dk per frame.  Blocks
    of 4800 samples (40 frames) carry the state; results are bit for bit the
    same alone and in the mix, and match the oracle's Eq. 5 / Eqs. 11-12 on
    its own interpolation and step-up, with dL/dk by its chain rule."""
    hop = 120
    lengths = [4800, 0, 1, 17, 12000, 30001, 9600, 999, 20000, 121, 7000, 4799, 2400, 5001]
    kinds = [0, 0, 0, 1, 0, 1, 0, 1, 0, 0, 1, 0, 1, 0]
    rng = np.random.default_rng(8)
    reqs = []
    for T, kind in zip(lengths, kinds):
        k = inputs.reflection_frames(rng, 1, O.n_frames(T, hop), M, 0.95, 0.9)[0].astype(np.float32)
        e = rng.standard_normal(T).astype(np.float32)
        gs = rng.standard_normal(T).astype(np.float32) if kind else None
        reqs.append((torch.from_numpy(k).pin_memory(), torch.from_numpy(e).pin_memory(),
                     None if gs is None else torch.from_numpy(gs).pin_memory()))
    cfg = dict(CFG, block_rows=4800, hop=hop)
    with serve.Server(M, **cfg) as srv:
        mix = []
        for k, e, gs in reqs:
            mix.append(srv.submit(k, e, gs))
            time.sleep(float(rng.uniform(0, 3e-4)))
        srv.drain(timeout_s=60)
        st = srv.stats()
        alone = []
        for k, e, gs in reqs:
            alone.append(srv.submit(k, e, gs))
            srv.drain(timeout_s=60)
        assert _lib.lp_tv_device_status() == 0
    assert st["carried_blocks"] > 0 and st["max_signals_iter"] > 1 and st["adapt_calls"] > 0 and st["error"] == 0
    for x, y, (k, e, gs), T in zip(mix, alone, reqs, lengths):
        assert x.status == 0
        for u, v in zip(_outputs(x), _outputs(y)):
            assert np.array_equal(u, v), T
        if T == 0:
            continue
        a = O.coeffs(k.numpy(), T, hop)
        if gs is None:
            rs = O.forward(a, e.numpy())
            assert norm_err(x.s.numpy()[None], rs[None]).max() <= TOL_F32, T
        else:
            rs, rge, rga, _ = O.forward_backward(a[None], e.numpy()[None], gs.numpy()[None])
            rgk = O.coeffs_adjoint(k.numpy(), rga[0], hop)
            for name, got, ref in (("s", x.s, rs), ("ge", x.ge, rge), ("gk", x.ga, rgk[None])):
                err = norm_err(got.numpy().reshape(1, -1), ref.reshape(1, -1))
                assert err.max() <= TOL_F32, (name, T, err)
