"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function include/*.h declares.  Host-only entry points (error
strings, chunk and workspace queries, argument checks) are exercised; no
call here launches a kernel."""
from __future__ import annotations

import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2406_05128_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_\w+)\s*\(", text)))


def test_header_lists_match_binding():
    from paper_2406_05128_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_entry_points(lib):
    from paper_2406_05128_gb300 import _lib
    assert "sm_103a" in _lib.version()
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert _lib.strerror(code)
    assert "unknown" not in _lib.strerror(_lib.LP_ENONFINITE).lower()
    # argument checks of the non-finite check come before any CUDA call
    assert lib.lp_tv_check_finite_f32(None, 0, None) == _lib.LP_OK
    assert lib.lp_tv_check_finite_f32(None, 5, None) == _lib.LP_EINVAL
    assert lib.lp_tv_check_finite_f32(2, 5, None) == _lib.LP_EALIGN
    assert lib.lp_tv_check_finite_f64(4, 5, None) == _lib.LP_EALIGN
    L = _lib.lp_tv_pick_chunk(32, 48000, 22)
    assert L > 0 and L % 16 == 0
    assert _lib.lp_tv_num_chunks(48000, 22, L) == -(-48000 // L)
    assert _lib.lp_tv_workspace_bytes(32, 48000, 22, L) > 0
    assert _lib.lp_tv_workspace_bytes(-1, 10, 2) == 0
    assert _lib.lp_tv_workspace_bytes(2, 10, 40) == 0  # order above 32


def test_frames_row_cache_sizes(lib):
    """The cached frames workspace adds 4*M bytes per sample (256-aligned)
    for the compiled orders and nothing for padded ones."""
    from paper_2406_05128_gb300 import _lib
    for B, T, M, hop in ((32, 48000, 22, 120), (3, 1237, 16, 120), (2, 999, 13, 7), (1, 50, 8, 120)):
        n0 = _lib.lp_tv_workspace_bytes_frames(B, T, M, hop)
        n1 = _lib.lp_tv_workspace_bytes_frames_cached(B, T, M, hop)
        assert n0 > 0
        if M in (2, 4, 8, 12, 16, 22, 30, 32):
            assert n1 == n0 + ((B * T * M * 4 + 255) // 256) * 256
        else:
            assert n1 == n0
    assert _lib.lp_tv_workspace_bytes_frames_cached(2, 100, 4, 0) == 0  # hop < 1
    assert _lib.lp_tv_workspace_bytes_frames_cached(2, 100, 40, 10) == 0  # order above 32
    # varlen: the cache adds 4*M bytes per packed row (256-aligned) on top of
    # the workspace of a backward with dL/dk
    for n, total, M, frames in ((8, 12258, 22, 110), (3, 4000, 16, 40), (5, 999, 13, 30)):
        n0 = _lib.lp_tv_workspace_bytes_frames_varlen(n, total, M, frames)
        n1 = _lib.lp_tv_workspace_bytes_frames_varlen_cached(n, total, M, frames)
        assert n0 > 0
        if M in (2, 4, 8, 12, 16, 22, 30, 32):
            assert n1 == n0 + ((total * M * 4 + 255) // 256) * 256
        else:
            assert n1 == n0
    assert _lib.lp_tv_workspace_bytes_frames_varlen_cached(2, 100, 4, -1) == 0  # negative frame count


def test_argument_errors_without_launching(lib):
    from paper_2406_05128_gb300 import _lib
    f = lib.lp_tv_forward_f32
    assert f(-1, 10, 2, None, None, None, None, None, 0, 0, None, 0, None) == _lib.LP_EINVAL
    assert f(2, 10, 40, 8, 8, None, 8, None, 0, 0, None, 0, None) == _lib.LP_EUNSUPPORTED
    assert f(2, 10, 4, 16, None, None, 16, None, 0, 0, None, 0, None) == _lib.LP_EINVAL   # e NULL
    assert f(2, 10, 4, 16, 16, None, 16, None, 0, 7, None, 0, None) == _lib.LP_EINVAL     # bad algo
    assert f(2, 10, 4, 16, 16, None, 16, None, 0, 0, None, 0, None) == _lib.LP_EWORKSPACE  # no workspace
    assert f(2, 10, 4, 20, 16, None, 16, None, 0, 0, None, 0, None) == _lib.LP_EALIGN     # a misaligned
    assert f(0, 10, 4, None, None, None, None, None, 0, 0, None, 0, None) == _lib.LP_OK   # empty batch
    g = lib.lp_tv_backward_f64
    assert g(2, 10, 40, 8, 8, 8, None, 8, None, None, 0, 0, 0, None, 0, None) == _lib.LP_EUNSUPPORTED  # f64: M <= 16
    assert g(2, 10, 4, 16, 16, None, None, 16, 16, None, 0, 0, 0, None, 0, None) == _lib.LP_EINVAL  # ga needs s
    assert g(2, 10, 4, 16, 16, 16, None, 16, None, None, 0, 0, 4, None, 0, None) == _lib.LP_EINVAL  # bad flag
    # LP_BWD_FUSED_GA is accepted (then the missing workspace is the error)
    assert g(2, 10, 4, 16, 16, 16, None, 16, 16, None, 0, 0, 3, None, 0, None) == _lib.LP_EWORKSPACE


def test_serve_host_only_entry_points(lib):
    """Configuration checks of the serving loop run before any CUDA call."""
    from paper_2406_05128_gb300 import _lib
    cfg = _lib.ServeConfig()
    lib.lp_serve_default_config(ctypes.byref(cfg))
    assert (cfg.M, cfg.block_rows, cfg.max_signals, cfg.max_inflight) == (22, 96000, 256, 4)
    assert cfg.hbm_budget == 20 << 30
    h = ctypes.c_void_p()
    for field, bad in (("M", 0), ("M", 33), ("max_signals", 0), ("max_inflight", 0), ("max_inflight", 17),
                       ("block_rows", -2), ("max_iter_rows", 1)):
        c = _lib.ServeConfig()
        lib.lp_serve_default_config(ctypes.byref(c))
        setattr(c, field, bad)
        assert lib.lp_serve_create(ctypes.byref(c), ctypes.byref(h)) == _lib.LP_EINVAL, field
    c = _lib.ServeConfig()
    lib.lp_serve_default_config(ctypes.byref(c))
    c.chunk = 256
    c.hbm_budget = 64 << 20  # cannot hold one largest iteration of 4 M rows
    assert lib.lp_serve_create(ctypes.byref(c), ctypes.byref(h)) == _lib.LP_ETOOBIG
    assert lib.lp_serve_submit(None, 0, 0, 10, 8, 8, None, 8, None, None, 0) == _lib.LP_EINVAL
    t0 = lib.lp_serve_now_ns()
    assert lib.lp_serve_now_ns() >= t0 > 0


def test_selftest_rejects_unknown_wait_without_launching(lib):
    from paper_2406_05128_gb300 import _lib
    assert lib.lp_tv_selftest_wait(0, None) == _lib.LP_EINVAL
    assert lib.lp_tv_selftest_wait(3, None) == _lib.LP_EINVAL


def test_threads_per_chunk_arguments(lib):
    """The launch-shape setting (host only): defaults and the two
    alternatives are accepted, anything else is LP_EINVAL."""
    from paper_2406_05128_gb300 import _lib
    assert lib.lp_tv_set_threads_per_chunk(0, 0) == _lib.LP_OK
    assert lib.lp_tv_set_threads_per_chunk(2, 8) == _lib.LP_OK
    assert lib.lp_tv_set_threads_per_chunk(1, 16) == _lib.LP_OK
    assert lib.lp_tv_set_threads_per_chunk(3, 16) == _lib.LP_EINVAL
    assert lib.lp_tv_set_threads_per_chunk(1, 12) == _lib.LP_EINVAL
