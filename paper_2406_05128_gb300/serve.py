"""Serving loop: continuous batching of time-varying LP filter requests.

Binding of the C ABI in include/tvlp_serve.h (argument marshalling only; the
scheduling runs in the library's worker thread and every computation in its
CUDA kernels).  A request is one signal on the host: synthesis (Eq. 5,
s = LP_a(e)) or adaptation (Eq. 5 and its adjoint, Eq. 11 and Eq. 12: s, ge,
ga for a given gs).  Inputs are CPU float32 tensors, page-locked so that the
copies overlap with compute; outputs are allocated page-locked here.
"""
from __future__ import annotations

import ctypes
import itertools

import torch

from . import _lib

SYNTH = _lib.LP_SERVE_SYNTH
ADAPT = _lib.LP_SERVE_ADAPT


def now_ns() -> int:
    """The server's clock (monotonic nanoseconds)."""
    return _lib.load().lp_serve_now_ns()


class Request:
    """One submitted request: its inputs, outputs and, once polled, its
    latency (ns, arrival to results on the host) and status."""

    __slots__ = ("id", "kind", "T", "a", "e", "gs", "s", "ge", "ga", "latency_ns", "status", "tag")

    def __init__(self, rid, kind, a, e, gs, s, ge, ga, tag=None):
        self.id, self.kind, self.T = rid, kind, e.shape[0]
        self.a, self.e, self.gs, self.s, self.ge, self.ga = a, e, gs, s, ge, ga
        self.latency_ns = None
        self.status = None
        self.tag = tag

    @property
    def done(self) -> bool:
        return self.status is not None


def _host(x, name, shape):
    if not isinstance(x, torch.Tensor) or x.device.type != "cpu" or x.dtype != torch.float32:
        raise ValueError(f"{name} must be a CPU float32 tensor")
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {tuple(shape)}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return x


class Server:
    """A serving loop on one GPU (see include/tvlp_serve.h).

    M, chunk, block_rows, max_signals, max_iter_rows, max_inflight and
    hbm_budget are the fields of lp_serve_config; chunk=0 lets the library
    pick one chunk length for every call."""

    def __init__(self, M: int = 22, *, chunk: int = 0, block_rows: int = 96000, max_signals: int = 256,
                 max_iter_rows: int = 4 << 20, max_inflight: int = 4, hbm_budget: int = 20 << 30, hop: int = 0,
                 device=None, require_pinned: bool = True):
        lib = _lib.load()
        self._lib = lib
        cfg = _lib.ServeConfig()
        lib.lp_serve_default_config(ctypes.byref(cfg))
        cfg.M, cfg.chunk, cfg.block_rows = M, chunk, block_rows
        cfg.max_signals, cfg.max_iter_rows, cfg.max_inflight, cfg.hbm_budget = (max_signals, max_iter_rows,
                                                                                max_inflight, hbm_budget)
        cfg.hop = hop
        self.M = M
        self.hop = hop
        self.require_pinned = require_pinned
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("the serving loop runs on a CUDA device")
        self.device = dev
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _lib._check(lib.lp_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "lp_serve_create")
        self._h = h
        self._ids = itertools.count()
        self._pending: dict[int, Request] = {}
        n = 1024
        self._pid = (ctypes.c_int64 * n)()
        self._plat = (ctypes.c_int64 * n)()
        self._pst = (ctypes.c_int * n)()

    def submit(self, a, e, gs=None, *, arrival_ns: int = 0, out=None, tag=None) -> Request:
        """Queue one request.  a [T, M] (a server with hop > 0: reflection
        coefficients per frame, [ceil(T/hop)+1, M]), e [T] (and gs [T] for
        adaptation) are CPU float32 tensors; out optionally gives the output
        tensors (s, or (s, ge, ga); on a frames server ga is dL/dk per
        frame).  Returns the Request, whose outputs are valid once poll() has
        returned it."""
        if self._h is None:
            raise RuntimeError("server is closed")
        T = e.shape[0] if isinstance(e, torch.Tensor) else -1
        _host(e, "e", (T,))
        _host(a, "a", ((-(-T // self.hop) + 1) if self.hop > 0 else T, self.M))
        kind = ADAPT if gs is not None else SYNTH
        if gs is not None:
            _host(gs, "gs", (T,))
        if self.require_pinned and T > 0 and not all(x.is_pinned() for x in (a, e) + ((gs,) if gs is not None else ())):
            raise ValueError("inputs must be page-locked (tensor.pin_memory()) so the copies overlap with compute")
        # coefficient gradient rows: dL/da per sample, or dL/dk per frame
        cg_rows = (-(-T // self.hop) + 1) if self.hop > 0 else T
        if out is None:
            s = torch.empty((T,), dtype=torch.float32, pin_memory=True)
            ge = torch.empty((T,), dtype=torch.float32, pin_memory=True) if kind == ADAPT else None
            ga = torch.empty((cg_rows, self.M), dtype=torch.float32, pin_memory=True) if kind == ADAPT else None
        elif kind == ADAPT:
            s, ge, ga = out
            _host(ge, "ge", (T,))
            _host(ga, "ga", (cg_rows, self.M))
        else:
            s, ge, ga = (out[0] if isinstance(out, (tuple, list)) else out), None, None
        _host(s, "s", (T,))
        rid = next(self._ids)
        req = Request(rid, kind, a, e, gs, s, ge, ga, tag)
        p = lambda x: None if x is None else x.data_ptr()  # noqa: E731
        self._pending[rid] = req
        rc = self._lib.lp_serve_submit(self._h, rid, kind, T, p(a), p(e), p(gs), p(s), p(ge), p(ga), int(arrival_ns))
        if rc != _lib.LP_OK:
            del self._pending[rid]
            raise _lib.LPError(rc, "lp_serve_submit")
        return req

    def poll(self) -> list:
        """Requests completed since the last poll (never blocks)."""
        out = []
        while True:
            n = self._lib.lp_serve_poll(self._h, self._pid, self._plat, self._pst, len(self._pid))
            if n < 0:
                raise _lib.LPError(n, "lp_serve_poll")
            for k in range(n):
                req = self._pending.pop(self._pid[k])
                req.latency_ns, req.status = self._plat[k], self._pst[k]
                out.append(req)
            if n < len(self._pid):
                return out

    def drain(self, timeout_s: float | None = None) -> list:
        """Wait until every submitted request has completed; returns the
        ones not yet polled."""
        ms = -1 if timeout_s is None else int(timeout_s * 1000)
        rc = self._lib.lp_serve_drain(self._h, ms)
        done = self.poll()
        _lib._check(rc, "lp_serve_drain")
        return done

    def stats(self, reset: bool = False) -> dict:
        st = _lib.ServeStats()
        _lib._check(self._lib.lp_serve_stats_get(self._h, ctypes.byref(st), int(reset)), "lp_serve_stats_get")
        return st.as_dict()

    @property
    def pending(self) -> int:
        return len(self._pending)

    def close(self):
        if self._h is not None:
            rc = self._lib.lp_serve_destroy(self._h)
            self._h = None
            _lib._check(rc, "lp_serve_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None:
                self._lib.lp_serve_destroy(self._h)
        except Exception:
            pass
