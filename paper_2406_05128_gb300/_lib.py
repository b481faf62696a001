"""ctypes binding of libtvlp.so (the C ABI declared in include/tvlp.h and
include/tvlp_serve.h).

Argument marshalling only: every computation runs in the CUDA kernels of the
shared library.  Importing this module does not load the library; the first
call does, and raises LPLibraryMissing if it has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LP_OK = 0
LP_EINVAL = -1
LP_EUNSUPPORTED = -2
LP_EWORKSPACE = -3
LP_ECUDA = -4
LP_EALIGN = -5
LP_ETOOBIG = -6
LP_ETIMEOUT = -7
LP_ENONFINITE = -8
LP_NOALLOC_SCRATCH_BYTES = 32 << 20

LP_DTYPE_F32 = 0
LP_DTYPE_F64 = 1

LP_ALGO_CHUNKED = 0
LP_ALGO_PLAIN = 1

# Every function declared in include/*.h.
EXPORTS = (
    "lp_strerror", "lp_version", "lp_tv_pick_chunk", "lp_tv_num_chunks",
    "lp_tv_workspace_bytes", "lp_tv_forward_f32", "lp_tv_forward_f64",
    "lp_tv_backward_f32", "lp_tv_backward_f64", "lp_tv_set_profile_events",
    "lp_tv_device_status", "lp_tv_forward_noalloc_f32",
    "lp_tv_backward_recompute_f32", "lp_tv_backward_recompute_f64",
    "lp_tv_workspace_bytes_varlen", "lp_tv_forward_varlen_f32", "lp_tv_forward_varlen_f64",
    "lp_tv_backward_varlen_f32", "lp_tv_backward_varlen_f64",
    "lp_tv_workspace_bytes_frames", "lp_tv_workspace_bytes_frames_cached", "lp_tv_forward_frames_f32",
    "lp_tv_check_finite_f32", "lp_tv_check_finite_f64", "lp_tv_workspace_bytes_frames_varlen_cached", "lp_tv_backward_frames_f32",
    "lp_tv_forward_frames_varlen_f32", "lp_tv_selftest_wait", "lp_tv_workspace_bytes_frames_varlen",
    "lp_tv_backward_frames_varlen_f32", "lp_tv_l2_set_aside", "lp_tv_workspace_bytes_ti", "lp_tv_forward_ti_f32", "lp_tv_backward_ti_f32",
    "lp_serve_default_config", "lp_serve_create", "lp_serve_destroy", "lp_serve_submit",
    "lp_serve_poll", "lp_serve_drain", "lp_serve_stats_get", "lp_serve_now_ns",
    "lp_framewise_num_frames", "lp_framewise_outputs_bytes", "lp_framewise_forward_f32",
    "lp_framewise_backward_f32", "lp_tv_mixed_coeff_offsets", "lp_tv_workspace_bytes_mixed",
    "lp_tv_forward_mixed_f32", "lp_tv_backward_mixed_f32", "lp_tv_set_threads_per_chunk",
)

LP_SERVE_SYNTH = 0
LP_SERVE_ADAPT = 1


class ServeConfig(ctypes.Structure):
    """lp_serve_config (include/tvlp_serve.h)."""
    _fields_ = [("M", ctypes.c_int), ("chunk", ctypes.c_int), ("block_rows", ctypes.c_int64),
                ("max_signals", ctypes.c_int), ("max_iter_rows", ctypes.c_int64),
                ("max_inflight", ctypes.c_int), ("hbm_budget", ctypes.c_uint64), ("hop", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    """lp_serve_stats (include/tvlp_serve.h)."""
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "completed", "iterations", "synth_calls", "adapt_calls", "kernel_launches", "blocks",
        "carried_blocks", "rows", "max_signals_iter", "max_waiting", "overlapped")] + \
        [(n, ctypes.c_uint64) for n in ("device_bytes", "ring_bytes", "ring_peak")] + \
        [("chunk", ctypes.c_int), ("error", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}

LP_BWD_REUSE_FORWARD = 1
LP_BWD_FUSED_GA = 2


class LPLibraryMissing(RuntimeError):
    pass


class LPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


_lock = threading.Lock()
_lib = None


def _declare(lib):
    c = ctypes
    vp, sz, i32, i64 = c.c_void_p, c.c_size_t, c.c_int, c.c_int64
    lib.lp_strerror.argtypes = [i32]
    lib.lp_strerror.restype = c.c_char_p
    lib.lp_version.argtypes = []
    lib.lp_version.restype = c.c_char_p
    lib.lp_tv_pick_chunk.argtypes = [i32, i64, i32, i32]
    lib.lp_tv_pick_chunk.restype = i32
    lib.lp_tv_num_chunks.argtypes = [i64, i32, i32]
    lib.lp_tv_num_chunks.restype = i64
    lib.lp_tv_workspace_bytes.argtypes = [i32, i64, i32, i32, i32]
    lib.lp_tv_workspace_bytes.restype = sz
    for name in ("lp_tv_forward_f32", "lp_tv_forward_f64"):
        f = getattr(lib, name)
        f.argtypes = [i32, i64, i32, vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
        f.restype = i32
    for name in ("lp_tv_backward_f32", "lp_tv_backward_f64"):
        f = getattr(lib, name)
        f.argtypes = [i32, i64, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, vp, sz, vp]
        f.restype = i32
    for name in ("lp_tv_backward_recompute_f32", "lp_tv_backward_recompute_f64"):
        f = getattr(lib, name)
        f.argtypes = [i32, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
        f.restype = i32
    lib.lp_tv_workspace_bytes_varlen.argtypes = [i32, i64, i32, i32, i32]
    lib.lp_tv_workspace_bytes_varlen.restype = sz
    for name in ("lp_tv_forward_varlen_f32", "lp_tv_forward_varlen_f64"):
        f = getattr(lib, name)
        f.argtypes = [i32, vp, i64, i32, vp, vp, vp, vp, vp, i32, vp, sz, vp]
        f.restype = i32
    for name in ("lp_tv_backward_varlen_f32", "lp_tv_backward_varlen_f64"):
        f = getattr(lib, name)
        f.argtypes = [i32, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
        f.restype = i32
    lib.lp_tv_workspace_bytes_frames.argtypes = [i32, i64, i32, i32, i32]
    lib.lp_tv_workspace_bytes_frames.restype = sz
    lib.lp_tv_workspace_bytes_frames_cached.argtypes = [i32, i64, i32, i32, i32]
    lib.lp_tv_workspace_bytes_frames_cached.restype = sz
    for name in ("lp_tv_check_finite_f32", "lp_tv_check_finite_f64"):
        getattr(lib, name).argtypes = [vp, sz, vp]
        getattr(lib, name).restype = i32
    lib.lp_tv_forward_frames_f32.argtypes = [i32, i64, i32, i32, vp, vp, vp, vp, vp, i32, vp, sz, vp]
    lib.lp_tv_forward_frames_f32.restype = i32
    lib.lp_tv_backward_frames_f32.argtypes = [i32, i64, i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
    lib.lp_tv_backward_frames_f32.restype = i32
    lib.lp_tv_forward_frames_varlen_f32.argtypes = [i32, vp, i64, i32, i32, vp, vp, vp, vp, vp, vp, i32, vp, sz, vp]
    lib.lp_tv_forward_frames_varlen_f32.restype = i32
    lib.lp_tv_workspace_bytes_frames_varlen.argtypes = [i32, i64, i32, i64, i32]
    lib.lp_tv_workspace_bytes_frames_varlen.restype = sz
    lib.lp_tv_workspace_bytes_frames_varlen_cached.argtypes = [i32, i64, i32, i64, i32]
    lib.lp_tv_workspace_bytes_frames_varlen_cached.restype = sz
    lib.lp_tv_backward_frames_varlen_f32.argtypes = [i32, vp, i64, i32, i32, vp, i64, vp, vp, vp, vp, vp, vp, vp, i32,
                                                     i32, vp, sz, vp]
    lib.lp_tv_backward_frames_varlen_f32.restype = i32
    lib.lp_tv_l2_set_aside.argtypes = [sz, c.POINTER(sz)]
    lib.lp_tv_l2_set_aside.restype = i32
    lib.lp_tv_selftest_wait.argtypes = [i32, vp]
    lib.lp_tv_selftest_wait.restype = i32
    lib.lp_tv_workspace_bytes_ti.argtypes = [i32, i64, i32, i32]
    lib.lp_tv_workspace_bytes_ti.restype = sz
    lib.lp_tv_set_threads_per_chunk.argtypes = [i32, i32]
    lib.lp_tv_set_threads_per_chunk.restype = i32
    lib.lp_tv_mixed_coeff_offsets.argtypes = [i32, vp, vp, vp]
    lib.lp_tv_mixed_coeff_offsets.restype = i64
    lib.lp_tv_workspace_bytes_mixed.argtypes = [i32, vp, vp, i32]
    lib.lp_tv_workspace_bytes_mixed.restype = sz
    lib.lp_tv_forward_mixed_f32.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp, sz, vp]
    lib.lp_tv_forward_mixed_f32.restype = i32
    lib.lp_tv_backward_mixed_f32.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
    lib.lp_tv_backward_mixed_f32.restype = i32
    lib.lp_framewise_num_frames.argtypes = [i64, i32]
    lib.lp_framewise_num_frames.restype = i64
    lib.lp_framewise_outputs_bytes.argtypes = [i32, i64, i32]
    lib.lp_framewise_outputs_bytes.restype = sz
    lib.lp_framewise_forward_f32.argtypes = [i32, i64, i32, i32, vp, vp, vp, vp, vp]
    lib.lp_framewise_forward_f32.restype = i32
    lib.lp_framewise_backward_f32.argtypes = [i32, i64, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.lp_framewise_backward_f32.restype = i32
    lib.lp_tv_forward_ti_f32.argtypes = [i32, i64, i32, vp, vp, vp, vp, vp, i32, vp, sz, vp]
    lib.lp_tv_forward_ti_f32.restype = i32
    lib.lp_tv_backward_ti_f32.argtypes = [i32, i64, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
    lib.lp_tv_backward_ti_f32.restype = i32
    lib.lp_tv_forward_noalloc_f32.argtypes = [i32, i64, i32, vp, vp, vp, vp, vp]
    lib.lp_tv_forward_noalloc_f32.restype = i32
    lib.lp_tv_device_status.argtypes = [i32]
    lib.lp_tv_device_status.restype = i32
    lib.lp_tv_set_profile_events.argtypes = [c.POINTER(vp), i32]
    lib.lp_tv_set_profile_events.restype = i32
    lib.lp_serve_default_config.argtypes = [c.POINTER(ServeConfig)]
    lib.lp_serve_default_config.restype = None
    lib.lp_serve_create.argtypes = [c.POINTER(ServeConfig), c.POINTER(vp)]
    lib.lp_serve_create.restype = i32
    lib.lp_serve_destroy.argtypes = [vp]
    lib.lp_serve_destroy.restype = i32
    lib.lp_serve_submit.argtypes = [vp, i64, i32, i64, vp, vp, vp, vp, vp, vp, i64]
    lib.lp_serve_submit.restype = i32
    lib.lp_serve_poll.argtypes = [vp, c.POINTER(i64), c.POINTER(i64), c.POINTER(i32), i32]
    lib.lp_serve_poll.restype = i32
    lib.lp_serve_drain.argtypes = [vp, i64]
    lib.lp_serve_drain.restype = i32
    lib.lp_serve_stats_get.argtypes = [vp, c.POINTER(ServeStats), i32]
    lib.lp_serve_stats_get.restype = i32
    lib.lp_serve_now_ns.argtypes = []
    lib.lp_serve_now_ns.restype = i64
    return lib


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load (once) and return the ctypes handle of libtvlp.so: `path`, else
    the build named by the TVLP_LIBRARY environment variable (the checked
    build with index checks, build.build(checks=True), for tests), else the
    package's own build."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or os.environ.get("TVLP_LIBRARY") or _build.LIB
            if not os.path.exists(p):
                raise LPLibraryMissing(
                    f"{p} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                    "(needs nvcc for sm_103a)")
            _lib = _declare(ctypes.CDLL(p))
    return _lib


def strerror(code: int) -> str:
    return load().lp_strerror(code).decode()


def version() -> str:
    return load().lp_version().decode()


def lp_tv_pick_chunk(B: int, T: int, M: int, dtype: int = LP_DTYPE_F32) -> int:
    return load().lp_tv_pick_chunk(B, T, M, dtype)


def lp_tv_num_chunks(T: int, M: int, chunk: int) -> int:
    return load().lp_tv_num_chunks(T, M, chunk)


def lp_tv_workspace_bytes(B: int, T: int, M: int, chunk: int = 0, dtype: int = LP_DTYPE_F32) -> int:
    return load().lp_tv_workspace_bytes(B, T, M, chunk, dtype)


def lp_tv_set_profile_events(event_handles):
    """Install per-kernel timing events (list of 2*n raw cudaEvent_t handles
    as ints) for calls from this thread; None uninstalls."""
    if not event_handles:
        _check(load().lp_tv_set_profile_events(None, 0), "lp_tv_set_profile_events")
        return None
    arr = (ctypes.c_void_p * len(event_handles))(*event_handles)
    _check(load().lp_tv_set_profile_events(arr, len(event_handles) // 2), "lp_tv_set_profile_events")
    return arr  # keep alive while installed


def _check(rc: int, where: str):
    if rc != LP_OK:
        raise LPError(rc, where)


def lp_tv_forward(dtype: int, B, T, M, a, e, zi, s, ckpt, chunk, algo, ws, ws_bytes, stream):
    """Raw forward call; pointers are ints (device addresses) or None."""
    fn = load().lp_tv_forward_f32 if dtype == LP_DTYPE_F32 else load().lp_tv_forward_f64
    _check(fn(B, T, M, a, e, zi, s, ckpt, chunk, algo, ws, ws_bytes, stream), "lp_tv_forward")


def lp_tv_backward(dtype: int, B, T, M, gs, a, s, zi, ge, ga, gzi, chunk, algo, flags, ws, ws_bytes, stream):
    """Raw backward call; pointers are ints (device addresses) or None."""
    fn = load().lp_tv_backward_f32 if dtype == LP_DTYPE_F32 else load().lp_tv_backward_f64
    _check(fn(B, T, M, gs, a, s, zi, ge, ga, gzi, chunk, algo, flags, ws, ws_bytes, stream), "lp_tv_backward")


def lp_tv_backward_recompute(dtype: int, B, T, M, gs, a, e, ckpt, zi, s, ge, ga, gzi, chunk, flags, ws, ws_bytes,
                             stream):
    """Raw backward from chunk checkpoints (s is recomputed into `s`)."""
    fn = load().lp_tv_backward_recompute_f32 if dtype == LP_DTYPE_F32 else load().lp_tv_backward_recompute_f64
    _check(fn(B, T, M, gs, a, e, ckpt, zi, s, ge, ga, gzi, chunk, flags, ws, ws_bytes, stream),
           "lp_tv_backward_recompute")


def lp_tv_workspace_bytes_varlen(n, total, M, chunk=0, dtype=LP_DTYPE_F32):
    return load().lp_tv_workspace_bytes_varlen(n, total, M, chunk, dtype)


def lp_tv_forward_varlen(dtype: int, n, offsets, total, M, a, e, zi, s, ckpt, chunk, ws, ws_bytes, stream):
    """Raw varlen forward; `offsets` is a device pointer to n+1 int64."""
    fn = load().lp_tv_forward_varlen_f32 if dtype == LP_DTYPE_F32 else load().lp_tv_forward_varlen_f64
    _check(fn(n, offsets, total, M, a, e, zi, s, ckpt, chunk, ws, ws_bytes, stream), "lp_tv_forward_varlen")


def lp_tv_backward_varlen(dtype: int, n, offsets, total, M, gs, a, s, zi, ge, ga, gzi, chunk, flags, ws, ws_bytes,
                          stream):
    """Raw varlen backward; `offsets` is a device pointer to n+1 int64."""
    fn = load().lp_tv_backward_varlen_f32 if dtype == LP_DTYPE_F32 else load().lp_tv_backward_varlen_f64
    _check(fn(n, offsets, total, M, gs, a, s, zi, ge, ga, gzi, chunk, flags, ws, ws_bytes, stream),
           "lp_tv_backward_varlen")


def lp_tv_forward_noalloc_f32(B, T, M, a, e, zi, s, stream):
    """Raw allocation-free forward call (FP32); pointers are ints or None."""
    _check(load().lp_tv_forward_noalloc_f32(B, T, M, a, e, zi, s, stream), "lp_tv_forward_noalloc_f32")


def lp_tv_device_status(reset: bool = False) -> int:
    """Status word of the current device (0 = every bounded wait completed)."""
    rc = load().lp_tv_device_status(1 if reset else 0)
    if rc < 0:
        raise LPError(rc, "lp_tv_device_status")
    return rc


def lp_tv_workspace_bytes_frames(B, T, M, hop, chunk=0):
    return load().lp_tv_workspace_bytes_frames(B, T, M, hop, chunk)


def lp_tv_workspace_bytes_frames_cached(B, T, M, hop, chunk=0):
    return load().lp_tv_workspace_bytes_frames_cached(B, T, M, hop, chunk)


def lp_tv_check_finite(dtype: int, x, n, stream) -> bool:
    """True if the n values at device address x are all finite (synchronises
    the stream); raises on any other error."""
    fn = load().lp_tv_check_finite_f32 if dtype == LP_DTYPE_F32 else load().lp_tv_check_finite_f64
    rc = fn(x, n, stream)
    if rc == LP_ENONFINITE:
        return False
    _check(rc, "lp_tv_check_finite")
    return True


def lp_tv_forward_frames(B, T, M, hop, k, e, zi, s, ckpt, chunk, ws, ws_bytes, stream):
    _check(load().lp_tv_forward_frames_f32(B, T, M, hop, k, e, zi, s, ckpt, chunk, ws, ws_bytes, stream),
           "lp_tv_forward_frames_f32")


def lp_tv_backward_frames(B, T, M, hop, gs, k, s, zi, ge, gk, gzi, chunk, flags, ws, ws_bytes, stream):
    _check(load().lp_tv_backward_frames_f32(B, T, M, hop, gs, k, s, zi, ge, gk, gzi, chunk, flags, ws, ws_bytes,
                                            stream), "lp_tv_backward_frames_f32")


def lp_tv_forward_frames_varlen(n, offsets, total, M, hop, frame_offsets, k, e, zi, s, ckpt, chunk, ws, ws_bytes,
                                stream):
    _check(load().lp_tv_forward_frames_varlen_f32(n, offsets, total, M, hop, frame_offsets, k, e, zi, s, ckpt, chunk,
                                                  ws, ws_bytes, stream), "lp_tv_forward_frames_varlen_f32")


def lp_tv_workspace_bytes_ti(B, T, M, chunk=0):
    return load().lp_tv_workspace_bytes_ti(B, T, M, chunk)


def lp_tv_forward_ti(B, T, M, a, e, zi, s, ckpt, chunk, ws, ws_bytes, stream):
    _check(load().lp_tv_forward_ti_f32(B, T, M, a, e, zi, s, ckpt, chunk, ws, ws_bytes, stream),
           "lp_tv_forward_ti_f32")


def lp_tv_backward_ti(B, T, M, gs, a, s, zi, ge, ga, gzi, chunk, flags, ws, ws_bytes, stream):
    _check(load().lp_tv_backward_ti_f32(B, T, M, gs, a, s, zi, ge, ga, gzi, chunk, flags, ws, ws_bytes, stream),
           "lp_tv_backward_ti_f32")


def lp_tv_workspace_bytes_frames_varlen(n, total, M, total_frames, chunk=0):
    return load().lp_tv_workspace_bytes_frames_varlen(n, total, M, total_frames, chunk)


def lp_tv_workspace_bytes_frames_varlen_cached(n, total, M, total_frames, chunk=0):
    return load().lp_tv_workspace_bytes_frames_varlen_cached(n, total, M, total_frames, chunk)


def lp_tv_backward_frames_varlen(n, offsets, total, M, hop, frame_offsets, total_frames, gs, k, s, zi, ge, gk, gzi,
                                 chunk, flags, ws, ws_bytes, stream):
    _check(load().lp_tv_backward_frames_varlen_f32(n, offsets, total, M, hop, frame_offsets, total_frames, gs, k, s,
                                                   zi, ge, gk, gzi, chunk, flags, ws, ws_bytes, stream),
           "lp_tv_backward_frames_varlen_f32")


def lp_tv_l2_set_aside(nbytes: int) -> int:
    """Set the current context's persisting L2 size (clipped to the device's
    maximum); returns the size applied."""
    got = ctypes.c_size_t()
    _check(load().lp_tv_l2_set_aside(int(nbytes), ctypes.byref(got)), "lp_tv_l2_set_aside")
    return got.value


def lp_framewise_num_frames(T: int, hop: int) -> int:
    return load().lp_framewise_num_frames(T, hop)


def lp_framewise_outputs_bytes(B: int, T: int, hop: int) -> int:
    return load().lp_framewise_outputs_bytes(B, T, hop)


def lp_framewise_forward(B, T, M, hop, af, e, s, y, stream):
    _check(load().lp_framewise_forward_f32(B, T, M, hop, af, e, s, y, stream), "lp_framewise_forward_f32")


def lp_framewise_backward(B, T, M, hop, af, y, gs, ge, gaf, stream):
    _check(load().lp_framewise_backward_f32(B, T, M, hop, af, y, gs, ge, gaf, stream), "lp_framewise_backward_f32")


def lp_tv_mixed_coeff_offsets(n, offsets_host, orders_host, aoff_host):
    """offsets_host / orders_host / aoff_host: addresses of HOST arrays."""
    return load().lp_tv_mixed_coeff_offsets(n, offsets_host, orders_host, aoff_host)


def lp_tv_workspace_bytes_mixed(n, offsets_host, orders_host, chunk=0):
    return load().lp_tv_workspace_bytes_mixed(n, offsets_host, orders_host, chunk)


def lp_tv_forward_mixed(n, offsets, orders, offsets_host, orders_host, a, e, zi, s, chunk, ws, ws_bytes, stream):
    _check(load().lp_tv_forward_mixed_f32(n, offsets, orders, offsets_host, orders_host, a, e, zi, s, chunk, ws,
                                          ws_bytes, stream), "lp_tv_forward_mixed_f32")


def lp_tv_backward_mixed(n, offsets, orders, offsets_host, orders_host, gs, a, s, zi, ge, ga, gzi, chunk, flags, ws,
                         ws_bytes, stream):
    _check(load().lp_tv_backward_mixed_f32(n, offsets, orders, offsets_host, orders_host, gs, a, s, zi, ge, ga, gzi,
                                           chunk, flags, ws, ws_bytes, stream), "lp_tv_backward_mixed_f32")


def lp_tv_set_threads_per_chunk(k1_lane_factor: int = 1, rerun_chunks_per_warp: int = 16):
    _check(load().lp_tv_set_threads_per_chunk(k1_lane_factor, rerun_chunks_per_warp), "lp_tv_set_threads_per_chunk")
