"""Autotuner of the chunk length and of the threads per signal.

The chunk length L sets how a batch maps onto the GPU: the summary kernel
runs one lane group per chunk, the re-run kernels one lane per chunk, and
the scan composes and chains about sqrt(nC/4)-chunk groups.  Longer chunks
mean fewer lanes and a shorter scan; shorter chunks the opposite.  The
threads per signal are set beside it (lp_tv_set_threads_per_chunk): the
summary kernel's lanes per chunk (the default packing or twice the lanes,
each with half the recursions) and the re-run kernels' chunks per warp (16
or 8).  The library's cost model picks L without running anything
(lp_tv_pick_chunk).  This module picks by timing: for a batch shape
(uniform B x T, or varlen lengths) and order M it runs forward + adjoint
for candidate L (multiples of 16 around the model's pick) on synthetic
inputs and keeps the fastest, then, with shapes=True, times the launch
shapes at that L and keeps the fastest of those.  Results are cached per
shape in the process.  A chosen launch shape applies to the calls made
afterwards from the same thread; use_shape() sets it for a block of code.
"""
from __future__ import annotations

import contextlib
import statistics

import torch

from . import _lib, ops

_CACHE: dict = {}

# (summary lanes-per-chunk factor, re-run chunks per warp); the first is the default
SHAPES = ((1, 16), (2, 16), (1, 8), (2, 8))


@contextlib.contextmanager
def use_shape(shape):
    """Calls made inside the block (from this thread) use launch shape `shape`."""
    _lib.lp_tv_set_threads_per_chunk(*shape)
    try:
        yield
    finally:
        _lib.lp_tv_set_threads_per_chunk(*SHAPES[0])


def _pick_shape(step, iters):
    res = {}
    for sh in SHAPES:
        with use_shape(sh):
            res[sh] = _time(step, iters)
    return min(res, key=res.get), res


def _candidates(pick: int, lo: int = 32, hi: int = 1024):
    c = {pick}
    for f in (0.5, 0.625, 0.75, 0.875, 1.25, 1.5, 2.0):
        c.add(int(round(pick * f / 16)) * 16)
    return sorted(x for x in c if lo <= x <= hi)


def _time(fn, iters: int, warmup: int = 2) -> float:
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for i in range(warmup + iters):
        ev0.record()
        fn()
        ev1.record()
        ev1.synchronize()
        if i >= warmup:
            times.append(ev0.elapsed_time(ev1))
    return statistics.median(times)


def tune_uniform(B: int, T: int, M: int, *, device="cuda", iters: int = 5, candidates=None, fwd_bwd: bool = True,
                 shapes: bool = False):
    """Fastest chunk length for a uniform B x T batch at order M: (L, {L: ms});
    with shapes=True, (L, launch shape, {L: ms}, {shape: ms})."""
    key = ("uniform", B, T, M, fwd_bwd, shapes)
    if key in _CACHE:
        return _CACHE[key]
    pick = _lib.lp_tv_pick_chunk(B, T, M)
    cands = candidates or _candidates(pick)
    g = torch.Generator(device=device)
    g.manual_seed(0)
    a = 0.01 * torch.randn((B, T, M), generator=g, device=device)
    e = torch.randn((B, T), generator=g, device=device)
    gs = torch.randn((B, T), generator=g, device=device)
    res = {}
    for L in cands:
        ws = ops.workspace(B, T, M, L, torch.float32, device)

        def step():
            s = ops.lp_tv_forward(a, e, chunk=L, ws=ws)
            if fwd_bwd:
                ops.lp_tv_backward(gs, a, s, chunk=L, ws=ws, reuse_forward=True, need_gzi=False)

        res[L] = _time(step, iters)
    best = min(res, key=res.get)
    if shapes:
        ws = ops.workspace(B, T, M, best, torch.float32, device)

        def step_best():
            s = ops.lp_tv_forward(a, e, chunk=best, ws=ws)
            if fwd_bwd:
                ops.lp_tv_backward(gs, a, s, chunk=best, ws=ws, reuse_forward=True, need_gzi=False)

        shape, res_sh = _pick_shape(step_best, iters)
        _CACHE[key] = (best, shape, res, res_sh)
        return _CACHE[key]
    _CACHE[key] = (best, res)
    return best, res


def tune_varlen(lengths, M: int, *, device="cuda", iters: int = 5, candidates=None, fwd_bwd: bool = True,
                shapes: bool = False):
    """Fastest chunk length for a varlen batch with these signal lengths at
    order M: (L, {L: ms}); with shapes=True, (L, launch shape, {L: ms},
    {shape: ms})."""
    lengths = [int(x) for x in lengths]
    key = ("varlen", tuple(lengths), M, fwd_bwd, shapes)
    if key in _CACHE:
        return _CACHE[key]
    pk = ops.Packed(lengths, device)
    n = max(pk.n, 1)
    pick = _lib.lp_tv_pick_chunk(n, -(-pk.total // n), M)
    cands = candidates or _candidates(pick)
    g = torch.Generator(device=device)
    g.manual_seed(0)
    a = 0.01 * torch.randn((pk.total, M), generator=g, device=device)
    e = torch.randn((pk.total,), generator=g, device=device)
    gs = torch.randn((pk.total,), generator=g, device=device)
    res = {}
    for L in cands:
        nb = _lib.lp_tv_workspace_bytes_varlen(pk.n, pk.total, M, L)
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=device)

        def step():
            s = ops.lp_tv_forward_varlen(pk, a, e, chunk=L, ws=ws)
            if fwd_bwd:
                ops.lp_tv_backward_varlen(pk, gs, a, s, chunk=L, ws=ws, reuse_forward=True, need_gzi=False)

        res[L] = _time(step, iters)
    best = min(res, key=res.get)
    if shapes:
        nb = _lib.lp_tv_workspace_bytes_varlen(pk.n, pk.total, M, best)
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=device)

        def step_best():
            s = ops.lp_tv_forward_varlen(pk, a, e, chunk=best, ws=ws)
            if fwd_bwd:
                ops.lp_tv_backward_varlen(pk, gs, a, s, chunk=best, ws=ws, reuse_forward=True, need_gzi=False)

        shape, res_sh = _pick_shape(step_best, iters)
        _CACHE[key] = (best, shape, res, res_sh)
        return _CACHE[key]
    _CACHE[key] = (best, res)
    return best, res
