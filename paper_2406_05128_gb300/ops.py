"""PyTorch front end of the time-varying LP library.

PyTorch supplies device memory and the current CUDA stream; every step of
the filter, its adjoint and the coefficient gradient runs in libtvlp.so.
There is no CPU path: tensors must live on a CUDA device, and a missing
library raises instead of falling back.

    s = lp_filter(a, e, zi=None)          # differentiable, Eq. 5
    s = lp_tv_forward(a, e, zi)            # plain call
    ge, ga, gzi = lp_tv_backward(gs, a, s, zi)
"""
from __future__ import annotations

import torch

from . import _lib

_ALGOS = {"chunked": _lib.LP_ALGO_CHUNKED, "plain": _lib.LP_ALGO_PLAIN}


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return _lib.LP_DTYPE_F32
    if t.dtype == torch.float64:
        return _lib.LP_DTYPE_F64
    raise TypeError(f"unsupported dtype {t.dtype}; use float32 or float64")


def _check(t, name, shape, dtype, device):
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if t.dtype != dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


def all_finite(t: torch.Tensor) -> bool:
    """True if every element of the CUDA tensor t (float32 or float64,
    contiguous) is finite: one pass in the library's check kernel, then a
    synchronisation of the current stream (lp_tv_check_finite_*)."""
    _check(t, "t", tuple(t.shape), t.dtype, t.device)
    with torch.cuda.device(t.device):
        return _lib.lp_tv_check_finite(_dtype_code(t), t.data_ptr(), t.numel(), _stream(t.device))


def workspace(B: int, T: int, M: int, chunk: int = 0, dtype=torch.float32, device=None) -> torch.Tensor:
    """Workspace tensor (uint8) sized for one forward or backward call."""
    code = _lib.LP_DTYPE_F32 if dtype == torch.float32 else _lib.LP_DTYPE_F64
    n = _lib.lp_tv_workspace_bytes(B, T, M, chunk, code)
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device)


def lp_tv_forward(a, e, zi=None, *, chunk: int = 0, algo: str = "chunked", ckpt: bool = False, ws=None):
    """s(t) = e(t) - sum_i a_i(t) s(t-i)  (Eq. 5), batched.

    a [B,T,M], e [B,T], zi [B,M] or None (zi[:, j-1] = s(-j)).
    Returns s, or (s, ckpt) with ckpt [B, nC, M] the incoming state of every
    chunk when ckpt=True.
    """
    B, T, M = a.shape
    dev = a.device
    _check(a, "a", (B, T, M), a.dtype, dev)
    _check(e, "e", (B, T), a.dtype, dev)
    _check(zi, "zi", (B, M), a.dtype, dev)
    code = _dtype_code(a)
    with torch.cuda.device(dev):
        s = torch.empty((B, T), dtype=a.dtype, device=dev)
        ck = None
        if ckpt:
            nC = _lib.lp_tv_num_chunks(T, M, chunk or _lib.lp_tv_pick_chunk(B, T, M, code)) if M > 0 else 0
            ck = torch.empty((B, nC, M), dtype=a.dtype, device=dev)
        if ws is None:
            ws = workspace(B, T, M, chunk, a.dtype, dev)
        _lib.lp_tv_forward(code, B, T, M, _ptr(a), _ptr(e), _ptr(zi), _ptr(s), _ptr(ck), chunk,
                           _ALGOS[algo], _ptr(ws), ws.numel(), _stream(dev))
    return (s, ck) if ckpt else s


def _bwd_flags(reuse_forward: bool, fused_ga: bool) -> int:
    return (_lib.LP_BWD_REUSE_FORWARD if reuse_forward else 0) | (_lib.LP_BWD_FUSED_GA if fused_ga else 0)


def lp_tv_backward(gs, a, s, zi=None, *, need_ga: bool = True, need_gzi: bool = True, chunk: int = 0,
                   algo: str = "chunked", ws=None, reuse_forward: bool = False, fused_ga: bool = False):
    """Adjoint (Eqs. 11-12): returns (ge [B,T], ga [B,T,M] or None, gzi [B,M] or None).

    reuse_forward=True requires `ws` to be the workspace the forward call on
    the same `a` (and chunk) filled; the adjoint then reuses its chunk
    transfer matrices.  fused_ga=True has the adjoint re-run write ga
    instead of a pass of its own (same results).
    """
    B, T, M = a.shape
    dev = a.device
    _check(a, "a", (B, T, M), a.dtype, dev)
    _check(gs, "gs", (B, T), a.dtype, dev)
    _check(s, "s", (B, T), a.dtype, dev)
    _check(zi, "zi", (B, M), a.dtype, dev)
    code = _dtype_code(a)
    if reuse_forward and ws is None:
        raise ValueError("reuse_forward needs the forward's workspace")
    with torch.cuda.device(dev):
        ge = torch.empty((B, T), dtype=a.dtype, device=dev)
        ga = torch.empty((B, T, M), dtype=a.dtype, device=dev) if need_ga else None
        gzi = torch.empty((B, M), dtype=a.dtype, device=dev) if need_gzi else None
        if ws is None:
            ws = workspace(B, T, M, chunk, a.dtype, dev)
        flags = _bwd_flags(reuse_forward, fused_ga)
        _lib.lp_tv_backward(code, B, T, M, _ptr(gs), _ptr(a), _ptr(s), _ptr(zi), _ptr(ge), _ptr(ga), _ptr(gzi),
                            chunk, _ALGOS[algo], flags, _ptr(ws), ws.numel(), _stream(dev))
    return ge, ga, gzi


def lp_tv_backward_recompute(gs, a, e, ckpt, zi=None, *, need_ga: bool = True, need_gzi: bool = True,
                             chunk: int = 0, ws=None, reuse_forward: bool = False, fused_ga: bool = False):
    """Adjoint from chunk checkpoints: recomputes s from (a, e, ckpt) with
    the forward's chunk length, then returns (ge, ga or None, gzi or None)."""
    B, T, M = a.shape
    dev = a.device
    _check(a, "a", (B, T, M), a.dtype, dev)
    _check(gs, "gs", (B, T), a.dtype, dev)
    _check(e, "e", (B, T), a.dtype, dev)
    _check(zi, "zi", (B, M), a.dtype, dev)
    if ckpt is not None:
        _check(ckpt, "ckpt", tuple(ckpt.shape), a.dtype, dev)
    code = _dtype_code(a)
    with torch.cuda.device(dev):
        s = torch.empty((B, T), dtype=a.dtype, device=dev)
        ge = torch.empty((B, T), dtype=a.dtype, device=dev)
        ga = torch.empty((B, T, M), dtype=a.dtype, device=dev) if need_ga else None
        gzi = torch.empty((B, M), dtype=a.dtype, device=dev) if need_gzi else None
        if ws is None:
            ws = workspace(B, T, M, chunk, a.dtype, dev)
        flags = _bwd_flags(reuse_forward, fused_ga)
        _lib.lp_tv_backward_recompute(code, B, T, M, _ptr(gs), _ptr(a), _ptr(e), _ptr(ckpt), _ptr(zi), _ptr(s),
                                      _ptr(ge), _ptr(ga), _ptr(gzi), chunk, flags, _ptr(ws), ws.numel(),
                                      _stream(dev))
    return ge, ga, gzi


# ---------------------------------------------------------------------------
# Varlen batches: signals of different lengths packed back to back
# ---------------------------------------------------------------------------
class Packed:
    """Signals packed back to back for the varlen calls.

    rows [total] layout: signal b holds rows offsets[b] .. offsets[b] +
    lengths[b]; offsets are rounded up to even rows (16-byte aligned
    coefficient rows), the rows between signals are padding.  The library
    sees each signal as rows [offsets[b], offsets[b+1]) -- a signal followed
    by its padding, which comes after every real output and so leaves them
    unchanged; its inputs are zero.
    """

    def __init__(self, lengths, device, align: int = 2):
        self.lengths = [int(x) for x in lengths]
        starts, pos = [], 0
        for n in self.lengths:
            starts.append(pos)
            pos += n
            pos += (-pos) % align
        self.starts = starts
        self.total = pos
        self.n = len(self.lengths)
        self.offsets = torch.tensor(starts + [pos], dtype=torch.int64, device=device)
        self.device = device

    def pack(self, xs, width=None, dtype=torch.float32):
        """Concatenate per-signal tensors ([len] or [len, width]) into rows."""
        shape = (self.total,) if width is None else (self.total, width)
        out = torch.zeros(shape, dtype=dtype, device=self.device)
        for x, st, n in zip(xs, self.starts, self.lengths):
            out[st:st + n] = x
        return out

    def unpack(self, rows):
        return [rows[st:st + n] for st, n in zip(self.starts, self.lengths)]


def lp_tv_forward_varlen(packed: Packed, a, e, zi=None, *, chunk: int = 0, ckpt: bool = False, ws=None):
    """Forward filter (Eq. 5) over a varlen batch: a [total, M], e [total],
    zi [n, M] or None.  Returns s [total] (and the chunk checkpoints
    [nQ, M] with ckpt=True)."""
    total, M = a.shape
    dev = a.device
    _check(a, "a", (packed.total, M), a.dtype, dev)
    _check(e, "e", (packed.total,), a.dtype, dev)
    _check(zi, "zi", (packed.n, M), a.dtype, dev)
    code = _dtype_code(a)
    with torch.cuda.device(dev):
        s = torch.empty((total,), dtype=a.dtype, device=dev)
        ck = None
        if ckpt:
            L = chunk or _lib.lp_tv_pick_chunk(packed.n, -(-total // max(packed.n, 1)), M, code)
            L = -(-L // 16) * 16
            lens = (packed.offsets[1:] - packed.offsets[:-1]).tolist()
            nq = sum(-(-x // L) for x in lens)
            ck = torch.empty((nq, M), dtype=a.dtype, device=dev)
        if ws is None:
            nb = _lib.lp_tv_workspace_bytes_varlen(packed.n, total, M, chunk, code)
            ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        _lib.lp_tv_forward_varlen(code, packed.n, packed.offsets.data_ptr(), total, M, _ptr(a), _ptr(e), _ptr(zi),
                                  _ptr(s), _ptr(ck), chunk, _ptr(ws), ws.numel(), _stream(dev))
    return (s, ck) if ckpt else s


def lp_tv_backward_varlen(packed: Packed, gs, a, s, zi=None, *, need_ga: bool = True, need_gzi: bool = True,
                          chunk: int = 0, ws=None, reuse_forward: bool = False, fused_ga: bool = False):
    """Adjoint (Eqs. 11-12) over a varlen batch: returns (ge [total],
    ga [total, M] or None, gzi [n, M] or None)."""
    total, M = a.shape
    dev = a.device
    _check(gs, "gs", (total,), a.dtype, dev)
    _check(s, "s", (total,), a.dtype, dev)
    _check(zi, "zi", (packed.n, M), a.dtype, dev)
    code = _dtype_code(a)
    if reuse_forward and ws is None:
        raise ValueError("reuse_forward needs the forward's workspace")
    with torch.cuda.device(dev):
        ge = torch.empty((total,), dtype=a.dtype, device=dev)
        ga = torch.empty((total, M), dtype=a.dtype, device=dev) if need_ga else None
        gzi = torch.empty((packed.n, M), dtype=a.dtype, device=dev) if need_gzi else None
        if ws is None:
            nb = _lib.lp_tv_workspace_bytes_varlen(packed.n, total, M, chunk, code)
            ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        flags = _bwd_flags(reuse_forward, fused_ga)
        _lib.lp_tv_backward_varlen(code, packed.n, packed.offsets.data_ptr(), total, M, _ptr(gs), _ptr(a), _ptr(s),
                                   _ptr(zi), _ptr(ge), _ptr(ga), _ptr(gzi), chunk, flags, _ptr(ws), ws.numel(),
                                   _stream(dev))
    return ge, ga, gzi


class LPFunction(torch.autograd.Function):
    """Differentiable TV-LP filter: a non-differentiable fast kernel
    registered into the autograd graph with its adjoint (Sec. 2.2, Sec. 3.2).

    Default: the forward's output s and workspace (its chunk transfer
    matrices) are kept for the backward, which then runs one recursion per
    chunk.  With checkpoint=True only the per-chunk incoming states are kept
    (M values per chunk instead of s and the maps); the backward recomputes
    s from them and builds its own chunk maps."""

    @staticmethod
    def forward(ctx, a, e, zi, chunk, algo, checkpoint, check=False):
        a, e = a.contiguous(), e.contiguous()
        zi = zi.contiguous() if zi is not None else None
        B, T, M = a.shape
        ctx.chunk, ctx.algo, ctx.checkpoint = chunk, algo, bool(checkpoint and algo == "chunked" and M > 0)
        ctx.check = check
        if ctx.checkpoint:
            code = _dtype_code(a)
            ctx.chunk = chunk or _lib.lp_tv_pick_chunk(B, T, M, code)
            s, ck = lp_tv_forward(a, e, zi, chunk=ctx.chunk, algo=algo, ckpt=True)
            ctx.save_for_backward(a, e, zi, ck)
        else:
            ws = workspace(B, T, M, chunk, a.dtype, a.device)
            s = lp_tv_forward(a, e, zi, chunk=chunk, algo=algo, ws=ws)
            ctx.save_for_backward(a, s, zi, ws)
        if check:
            _raise_if_nonfinite(s, "s")
        return s

    @staticmethod
    def backward(ctx, gs):
        need_a, need_e, need_zi = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        if ctx.checkpoint:
            a, e, zi, ck = ctx.saved_tensors
            ge, ga, gzi = lp_tv_backward_recompute(gs.contiguous(), a, e, ck, zi, need_ga=need_a,
                                                   need_gzi=need_zi and zi is not None, chunk=ctx.chunk)
        else:
            a, s, zi, ws = ctx.saved_tensors
            ge, ga, gzi = lp_tv_backward(gs.contiguous(), a, s, zi, need_ga=need_a,
                                         need_gzi=need_zi and zi is not None, chunk=ctx.chunk, algo=ctx.algo,
                                         ws=ws, reuse_forward=ctx.algo == "chunked")
        if ctx.check:
            for name, g in (("dL/de", ge), ("dL/da", ga), ("dL/dzi", gzi)):
                if g is not None:
                    _raise_if_nonfinite(g, name)
        return (ga if need_a else None, ge if need_e else None, gzi if need_zi else None, None, None, None, None)


def _raise_if_nonfinite(t, name):
    if not all_finite(t):
        raise FloatingPointError(f"{name} holds an infinity or NaN (LP_ENONFINITE): a filter with a pole outside "
                                 "the unit circle, or a non-finite input")


def lp_filter(a, e, zi=None, *, chunk: int = 0, algo: str = "chunked", checkpoint: bool = False,
              check: bool = False):
    """Differentiable s = LP_{a(t)}(e) with optional initial state zi.
    checkpoint=True keeps per-chunk states instead of s for the backward.
    check=True raises FloatingPointError when s, or a gradient in the
    backward, holds an infinity or NaN (one extra pass and a stream
    synchronisation per tensor)."""
    return LPFunction.apply(a, e, zi, chunk, algo, checkpoint, check)


# ---------------------------------------------------------------------------
# Coefficients generated in the kernels (FP32): frame-rate reflection
# coefficients (Sec. 4.3) or one time-invariant row per signal (Eq. 2)
# ---------------------------------------------------------------------------
def n_frames(T: int, hop: int) -> int:
    """Frames of a T-sample signal at this hop: ceil(T / hop) + 1 (frame f
    sits at sample f * hop, and the last segment has an end frame)."""
    return -(-T // hop) + 1


def _f32(t, name):
    if t is not None and t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32 (generated coefficients are FP32)")


def workspace_frames(B: int, T: int, M: int, hop: int, chunk: int = 0, device=None,
                     cache_rows: bool = False) -> torch.Tensor:
    """Workspace of the frames calls.  cache_rows=True adds room for the
    generated rows (4*M bytes per sample, compiled orders only): the
    forward's first pass keeps them and the later passes stream them."""
    size = _lib.lp_tv_workspace_bytes_frames_cached if cache_rows else _lib.lp_tv_workspace_bytes_frames
    n = size(B, T, M, hop, chunk)
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device)


def workspace_ti(B: int, T: int, M: int, chunk: int = 0, device=None) -> torch.Tensor:
    n = _lib.lp_tv_workspace_bytes_ti(B, T, M, chunk)
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device)


def lp_tv_forward_frames(k, e, hop: int, zi=None, *, chunk: int = 0, ws=None):
    """Eq. 5 with a(t) generated in the kernels from k [B, F, M] (frame-rate
    reflection coefficients, F = ceil(T/hop)+1): interpolation per sample,
    then the step-up.  e [B, T]; returns s [B, T]."""
    B, F, M = k.shape
    T = e.shape[1]
    dev = k.device
    _f32(k, "k")
    _check(k, "k", (B, n_frames(T, hop), M), torch.float32, dev)
    _check(e, "e", (B, T), torch.float32, dev)
    _check(zi, "zi", (B, M), torch.float32, dev)
    with torch.cuda.device(dev):
        s = torch.empty((B, T), device=dev)
        if ws is None:
            ws = workspace_frames(B, T, M, hop, chunk, dev)
        _lib.lp_tv_forward_frames(B, T, M, hop, _ptr(k), _ptr(e), _ptr(zi), _ptr(s), None, chunk, _ptr(ws),
                                  ws.numel(), _stream(dev))
    return s


def lp_tv_backward_frames(gs, k, s, hop: int, zi=None, *, need_gk: bool = True, need_gzi: bool = True,
                          chunk: int = 0, ws=None, reuse_forward: bool = False):
    """Adjoint of lp_tv_forward_frames: (ge [B,T], gk [B,F,M] or None,
    gzi [B,M] or None).  reuse_forward: ws holds the forward's transfers."""
    B, F, M = k.shape
    T = gs.shape[1]
    dev = k.device
    _check(gs, "gs", (B, T), torch.float32, dev)
    _check(s, "s", (B, T), torch.float32, dev)
    _check(zi, "zi", (B, M), torch.float32, dev)
    with torch.cuda.device(dev):
        ge = torch.empty((B, T), device=dev)
        gk = torch.empty((B, F, M), device=dev) if need_gk else None
        gzi = torch.empty((B, M), device=dev) if need_gzi else None
        if ws is None:
            ws = workspace_frames(B, T, M, hop, chunk, dev)
        flags = _lib.LP_BWD_REUSE_FORWARD if reuse_forward else 0
        _lib.lp_tv_backward_frames(B, T, M, hop, _ptr(gs), _ptr(k), _ptr(s), _ptr(zi), _ptr(ge), _ptr(gk),
                                   _ptr(gzi), chunk, flags, _ptr(ws), ws.numel(), _stream(dev))
    return ge, gk, gzi


def lp_tv_forward_ti(a, e, zi=None, *, chunk: int = 0, ws=None):
    """Time-invariant filter (Eq. 2): a [B, M], one row per signal; e [B, T]."""
    B, M = a.shape
    T = e.shape[1]
    dev = a.device
    _check(a, "a", (B, M), torch.float32, dev)
    _check(e, "e", (B, T), torch.float32, dev)
    _check(zi, "zi", (B, M), torch.float32, dev)
    with torch.cuda.device(dev):
        s = torch.empty((B, T), device=dev)
        if ws is None:
            ws = workspace_ti(B, T, M, chunk, dev)
        _lib.lp_tv_forward_ti(B, T, M, _ptr(a), _ptr(e), _ptr(zi), _ptr(s), None, chunk, _ptr(ws), ws.numel(),
                              _stream(dev))
    return s


def lp_tv_backward_ti(gs, a, s, zi=None, *, need_ga: bool = True, need_gzi: bool = True, chunk: int = 0,
                      ws=None, reuse_forward: bool = False):
    """Adjoint of lp_tv_forward_ti: (ge [B,T], ga [B,M] = sum_t dL/da(t)
    (Eq. 3), gzi [B,M])."""
    B, M = a.shape
    T = gs.shape[1]
    dev = a.device
    _check(gs, "gs", (B, T), torch.float32, dev)
    _check(s, "s", (B, T), torch.float32, dev)
    with torch.cuda.device(dev):
        ge = torch.empty((B, T), device=dev)
        ga = torch.empty((B, M), device=dev) if need_ga else None
        gzi = torch.empty((B, M), device=dev) if need_gzi else None
        if ws is None:
            ws = workspace_ti(B, T, M, chunk, dev)
        flags = _lib.LP_BWD_REUSE_FORWARD if reuse_forward else 0
        _lib.lp_tv_backward_ti(B, T, M, _ptr(gs), _ptr(a), _ptr(s), _ptr(zi), _ptr(ge), _ptr(ga), _ptr(gzi), chunk,
                               flags, _ptr(ws), ws.numel(), _stream(dev))
    return ge, ga, gzi


class LPFramesFunction(torch.autograd.Function):
    """Differentiable filter with in-kernel coefficients from frame-rate
    reflection coefficients: gradients for k, e and zi."""

    @staticmethod
    def forward(ctx, k, e, zi, hop, chunk, cache_rows):
        k, e = k.contiguous(), e.contiguous()
        zi = zi.contiguous() if zi is not None else None
        B, F, M = k.shape
        ws = workspace_frames(B, e.shape[1], M, hop, chunk, k.device, cache_rows=cache_rows)
        s = lp_tv_forward_frames(k, e, hop, zi, chunk=chunk, ws=ws)
        ctx.hop, ctx.chunk = hop, chunk
        ctx.save_for_backward(k, s, zi, ws)
        return s

    @staticmethod
    def backward(ctx, gs):
        k, s, zi, ws = ctx.saved_tensors
        need_k, need_e, need_zi = ctx.needs_input_grad[:3]
        ge, gk, gzi = lp_tv_backward_frames(gs.contiguous(), k, s, ctx.hop, zi, need_gk=need_k,
                                            need_gzi=need_zi and zi is not None, chunk=ctx.chunk, ws=ws,
                                            reuse_forward=True)
        return (gk if need_k else None, ge if need_e else None, gzi if need_zi else None, None, None, None)


def lp_filter_frames(k, e, hop: int, zi=None, *, chunk: int = 0, cache_rows: bool = True):
    """Differentiable s = LP_{a(k)}(e) with a(t) generated in the kernels
    from frame-rate reflection coefficients k [B, ceil(T/hop)+1, M].
    cache_rows: keep the generated rows in the workspace between forward
    and backward (4*M bytes per sample) so that only the first pass
    generates them."""
    return LPFramesFunction.apply(k, e, zi, hop, chunk, cache_rows)


class LPTIFunction(torch.autograd.Function):
    """Differentiable time-invariant filter (Eq. 2) with GOLF's gradient (Eq. 3)."""

    @staticmethod
    def forward(ctx, a, e, zi, chunk):
        a, e = a.contiguous(), e.contiguous()
        zi = zi.contiguous() if zi is not None else None
        B, M = a.shape
        ws = workspace_ti(B, e.shape[1], M, chunk, a.device)
        s = lp_tv_forward_ti(a, e, zi, chunk=chunk, ws=ws)
        ctx.chunk = chunk
        ctx.save_for_backward(a, s, zi, ws)
        return s

    @staticmethod
    def backward(ctx, gs):
        a, s, zi, ws = ctx.saved_tensors
        need_a, need_e, need_zi = ctx.needs_input_grad[:3]
        ge, ga, gzi = lp_tv_backward_ti(gs.contiguous(), a, s, zi, need_ga=need_a,
                                        need_gzi=need_zi and zi is not None, chunk=ctx.chunk, ws=ws,
                                        reuse_forward=True)
        return (ga if need_a else None, ge if need_e else None, gzi if need_zi else None, None)


def lp_filter_ti(a, e, zi=None, *, chunk: int = 0):
    """Differentiable time-invariant all-pole filter, a [B, M]."""
    return LPTIFunction.apply(a, e, zi, chunk)


class PackedFrames:
    """Frames of a varlen batch.  The library gives signal b the frames of
    its whole slot of rows, [offsets[b], offsets[b+1]) of a Packed batch
    (the signal and its pad row): ceil(slot/hop)+1 frames, packed back to
    back from frame_offsets[b].  pack() repeats a signal's last frame where
    its slot needs one more than the signal itself."""

    def __init__(self, packed: Packed, hop: int):
        self.hop = hop
        ends = packed.starts[1:] + [packed.total]
        self.slots = [e - st for st, e in zip(packed.starts, ends)]
        self.counts = [n_frames(n, hop) for n in self.slots]
        starts, pos = [], 0
        for c in self.counts:
            starts.append(pos)
            pos += c
        self.starts, self.total = starts, pos
        self.offsets = torch.tensor(starts, dtype=torch.int64, device=packed.device)
        self.device = packed.device

    def pack(self, ks):
        """ks: per signal [n_frames(len_b, hop), M]."""
        rows = []
        for k, c in zip(ks, self.counts):
            k = k.reshape(k.shape[0], -1)
            if k.shape[0] < c:
                k = torch.cat([k, k[-1:].expand(c - k.shape[0], -1)])
            rows.append(k[:c])
        return torch.cat(rows).contiguous()


def lp_tv_forward_frames_varlen(packed: Packed, frames: PackedFrames, k, e, zi=None, *, chunk: int = 0, ws=None):
    """Varlen forward with generated coefficients: k [frames.total, M], e
    [packed.total]; returns s [packed.total]."""
    total = packed.total
    M = k.shape[1]
    dev = k.device
    _check(k, "k", (frames.total, M), torch.float32, dev)
    _check(e, "e", (total,), torch.float32, dev)
    _check(zi, "zi", (packed.n, M), torch.float32, dev)
    with torch.cuda.device(dev):
        s = torch.empty((total,), device=dev)
        if ws is None:
            nb = _lib.lp_tv_workspace_bytes_varlen(packed.n, total, M, chunk, _lib.LP_DTYPE_F32)
            ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        _lib.lp_tv_forward_frames_varlen(packed.n, packed.offsets.data_ptr(), total, M, frames.hop,
                                         frames.offsets.data_ptr(), _ptr(k), _ptr(e), _ptr(zi), _ptr(s), None, chunk,
                                         _ptr(ws), ws.numel(), _stream(dev))
    return s


def lp_tv_backward_frames_varlen(packed: Packed, frames: PackedFrames, gs, k, s, zi=None, *, need_gk: bool = True,
                                 need_gzi: bool = True, chunk: int = 0, ws=None, reuse_forward: bool = False):
    """Varlen adjoint with generated coefficients: (ge [total], gk
    [frames.total, M] or None, gzi [n, M] or None).  reuse_forward: ws holds
    the forward's transfers (then size it with
    lp_tv_workspace_bytes_frames_varlen)."""
    total = packed.total
    M = k.shape[1]
    dev = k.device
    _check(gs, "gs", (total,), torch.float32, dev)
    _check(s, "s", (total,), torch.float32, dev)
    _check(zi, "zi", (packed.n, M), torch.float32, dev)
    with torch.cuda.device(dev):
        ge = torch.empty((total,), device=dev)
        gk = torch.empty((frames.total, M), device=dev) if need_gk else None
        gzi = torch.empty((packed.n, M), device=dev) if need_gzi else None
        if ws is None:
            nb = _lib.lp_tv_workspace_bytes_frames_varlen(packed.n, total, M, frames.total, chunk)
            ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        flags = _lib.LP_BWD_REUSE_FORWARD if reuse_forward else 0
        _lib.lp_tv_backward_frames_varlen(packed.n, packed.offsets.data_ptr(), total, M, frames.hop,
                                          frames.offsets.data_ptr(), frames.total, _ptr(gs), _ptr(k), _ptr(s),
                                          _ptr(zi), _ptr(ge), _ptr(gk), _ptr(gzi), chunk, flags, _ptr(ws),
                                          ws.numel(), _stream(dev))
    return ge, gk, gzi


# ---------------------------------------------------------------------------
# Frame-wise overlap-add approximation (the GOLF-ff comparison of Sec. 4.3):
# per-frame time-invariant filters on Hann-windowed frames of 4*hop samples,
# one every hop samples, overlap-added (lp_framewise_* in include/tvlp.h).
# ---------------------------------------------------------------------------
def framewise_frames(T: int, hop: int) -> int:
    """Frames of the frame-wise approximation: ceil(T / hop) + 3."""
    return -(-T // hop) + 3


def lp_framewise_forward(af, e, hop: int, *, keep_outputs: bool = True):
    """s [B, T] from per-frame direct-form coefficients af [B, F, M] and e
    [B, T]; with keep_outputs also the frame outputs y [B, 4*hop, F] the
    backward needs.  Returns (s, y or None)."""
    B, F, M = af.shape
    T = e.shape[1]
    dev = af.device
    _check(af, "af", (B, framewise_frames(T, hop), M), torch.float32, dev)
    _check(e, "e", (B, T), torch.float32, dev)
    with torch.cuda.device(dev):
        s = torch.empty((B, T), device=dev)
        y = torch.empty((B, 4 * hop, F), device=dev) if keep_outputs else None
        _lib.lp_framewise_forward(B, T, M, hop, _ptr(af), _ptr(e), _ptr(s), _ptr(y), _stream(dev))
    return s, y


def lp_framewise_backward(gs, af, y, hop: int):
    """(ge [B, T], gaf [B, F, M]) for dL/ds = gs, from the forward's frame
    outputs y."""
    B, F, M = af.shape
    T = gs.shape[1]
    dev = af.device
    _check(gs, "gs", (B, T), torch.float32, dev)
    _check(af, "af", (B, framewise_frames(T, hop), M), torch.float32, dev)
    _check(y, "y", (B, 4 * hop, F), torch.float32, dev)
    with torch.cuda.device(dev):
        ge = torch.empty((B, T), device=dev)
        gaf = torch.empty((B, F, M), device=dev)
        _lib.lp_framewise_backward(B, T, M, hop, _ptr(af), _ptr(y), _ptr(gs), _ptr(ge), _ptr(gaf), _stream(dev))
    return ge, gaf


class LPFramewiseFunction(torch.autograd.Function):
    """Differentiable frame-wise approximation: gradients for af and e."""

    @staticmethod
    def forward(ctx, af, e, hop):
        af, e = af.contiguous(), e.contiguous()
        s, y = lp_framewise_forward(af, e, hop)
        ctx.hop = hop
        ctx.save_for_backward(af, y)
        return s

    @staticmethod
    def backward(ctx, gs):
        af, y = ctx.saved_tensors
        ge, gaf = lp_framewise_backward(gs.contiguous(), af, y, ctx.hop)
        need_af, need_e = ctx.needs_input_grad[:2]
        return (gaf if need_af else None, ge if need_e else None, None)


def lp_filter_framewise(af, e, hop: int):
    """Differentiable frame-wise overlap-add filter (not Eq. 5: each frame is
    filtered with its own time-invariant coefficients af [B, F, M])."""
    return LPFramewiseFunction.apply(af, e, hop)


# ---------------------------------------------------------------------------
# Mixed orders: signals of different lengths and orders in one call
# (lp_tv_*_mixed_f32 in include/tvlp.h).
# ---------------------------------------------------------------------------
class PackedMixed:
    """Layout of a mixed-order batch: rows of e, s, gs, ge back to back
    (signal b at rows offsets[b] .. offsets[b+1]), and each signal's
    coefficient rows of its own order M_b as one block of a flat array,
    starting at element aoff[b] (a multiple of 4).  Keeps host and device
    copies of the offsets and orders."""

    def __init__(self, lengths, orders, device):
        import numpy as np
        self.lengths = [int(x) for x in lengths]
        self.orders = [int(x) for x in orders]
        assert len(self.lengths) == len(self.orders)
        self.n = len(self.lengths)
        self.offsets_host = np.zeros(self.n + 1, dtype=np.int64)
        self.offsets_host[1:] = np.cumsum(self.lengths)
        self.orders_host = np.asarray(self.orders, dtype=np.int32)
        self.aoff = np.zeros(self.n + 1, dtype=np.int64)
        n_a = _lib.lp_tv_mixed_coeff_offsets(self.n, self.offsets_host.ctypes.data, self.orders_host.ctypes.data,
                                             self.aoff.ctypes.data)
        if n_a < 0:
            raise ValueError("invalid lengths or orders")
        self.total = int(self.offsets_host[-1])
        self.total_a = int(n_a)
        self.device = torch.device(device)
        self.offsets = torch.tensor(self.offsets_host, device=device)
        self.orders_dev = torch.tensor(self.orders_host, device=device)

    def pack_rows(self, xs):
        out = torch.zeros((self.total,), dtype=torch.float32, device=self.device)
        for x, st, n in zip(xs, self.offsets_host[:-1], self.lengths):
            out[int(st):int(st) + n] = x
        return out

    def unpack_rows(self, rows):
        return [rows[int(st):int(st) + n] for st, n in zip(self.offsets_host[:-1], self.lengths)]

    def pack_coeffs(self, xs):
        """Per-signal [len_b, M_b] tensors into the flat coefficient array."""
        out = torch.zeros((max(self.total_a, 1),), dtype=torch.float32, device=self.device)
        for x, ao, n, m in zip(xs, self.aoff[:-1], self.lengths, self.orders):
            out[int(ao):int(ao) + n * m] = x.reshape(-1)
        return out

    def unpack_coeffs(self, flat):
        return [flat[int(ao):int(ao) + n * m].reshape(n, m)
                for ao, n, m in zip(self.aoff[:-1], self.lengths, self.orders)]

    def workspace(self, chunk: int = 0):
        nb = _lib.lp_tv_workspace_bytes_mixed(self.n, self.offsets_host.ctypes.data, self.orders_host.ctypes.data,
                                              chunk)
        if nb == 0 and self.n > 0:
            raise ValueError("invalid mixed batch")
        return torch.empty(max(nb, 256), dtype=torch.uint8, device=self.device)


def lp_tv_forward_mixed(pm: PackedMixed, a, e, zi=None, *, chunk: int = 0, ws=None):
    """Eq. 5 for every signal of a mixed batch with its own order; a: the
    flat coefficient array, e: packed rows, zi: [n, 32] or None."""
    dev = pm.device
    _check(e, "e", (pm.total,), torch.float32, dev)
    _check(zi, "zi", (pm.n, 32), torch.float32, dev)
    with torch.cuda.device(dev):
        s = torch.empty((pm.total,), device=dev)
        if ws is None:
            ws = pm.workspace(chunk)
        _lib.lp_tv_forward_mixed(pm.n, _ptr(pm.offsets), _ptr(pm.orders_dev), pm.offsets_host.ctypes.data,
                                 pm.orders_host.ctypes.data, _ptr(a), _ptr(e), _ptr(zi), _ptr(s), chunk, _ptr(ws),
                                 ws.numel(), _stream(dev))
    return s


def lp_tv_backward_mixed(pm: PackedMixed, gs, a, s, zi=None, *, need_ga: bool = True, need_gzi: bool = True,
                         chunk: int = 0, ws=None, reuse_forward: bool = False):
    """(ge [total], ga (flat, like a) or None, gzi [n, 32] or None)."""
    dev = pm.device
    _check(gs, "gs", (pm.total,), torch.float32, dev)
    with torch.cuda.device(dev):
        ge = torch.empty((pm.total,), device=dev)
        ga = torch.zeros_like(a) if need_ga else None
        gzi = torch.zeros((pm.n, 32), device=dev) if need_gzi else None
        if ws is None:
            ws = pm.workspace(chunk)
            reuse_forward = False
        flags = _lib.LP_BWD_REUSE_FORWARD if reuse_forward else 0
        _lib.lp_tv_backward_mixed(pm.n, _ptr(pm.offsets), _ptr(pm.orders_dev), pm.offsets_host.ctypes.data,
                                  pm.orders_host.ctypes.data, _ptr(gs), _ptr(a), _ptr(s), _ptr(zi), _ptr(ge),
                                  _ptr(ga), _ptr(gzi), chunk, flags, _ptr(ws), ws.numel(), _stream(dev))
    return ge, ga, gzi
