"""The allocation-free forward entry point against the regular one.

lp_tv_forward_noalloc_f32 serves callers that cannot allocate device memory
when they run the filter (a real-time callback that must not wait on the
allocator, a plugin inside a host that owns the GPU memory).  It keeps the
scan's scratch in a fixed array inside the library; its results must match
lp_tv_forward_f32 within the parity tolerance, on consecutive calls that
reuse that array.  This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _noalloc(a, e, zi):
    B, T, M = a.shape
    s = torch.empty((B, T), device=DEV)
    _lib.lp_tv_forward_noalloc_f32(B, T, M, a.data_ptr(), e.data_ptr(), None if zi is None else zi.data_ptr(),
                                   s.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return s


def test_noalloc_matches_regular_forward_twice():
    # two different problems in a row: the second call reuses the array the
    # first one filled
    for seed, (B, T, M) in ((21, (4, 20000, 22)), (22, (3, 7777, 16))):
        w = inputs.make("noalloc", B, T, M, seed=seed, gen="stable", with_zi=True)
        a, e, zi = (torch.tensor(x, device=DEV) for x in (w.a, w.e, w.zi))
        want = ops.lp_tv_forward(a, e, zi)
        got = _noalloc(a, e, zi)
        torch.cuda.synchronize()
        err = norm_err(got.cpu().numpy(), want.cpu().numpy())
        assert err.max() <= TOL_F32, err


def test_noalloc_rejects_problems_beyond_its_scratch():
    B, T, M = 64, 200000, 22
    need = _lib.lp_tv_workspace_bytes(B, T, M)
    assert need > _lib.LP_NOALLOC_SCRATCH_BYTES
    with pytest.raises(_lib.LPError) as ei:
        _lib.lp_tv_forward_noalloc_f32(B, T, M, 16, 16, None, 16, None)  # rejected before any use of the pointers
    assert ei.value.code == _lib.LP_ETOOBIG


def test_noalloc_without_initial_state_and_order_zero():
    w = inputs.make("noalloc0", 2, 5000, 12, seed=23, gen="stable")
    a, e = (torch.tensor(x, device=DEV) for x in (w.a, w.e))
    want = ops.lp_tv_forward(a, e)
    got = _noalloc(a, e, None)
    torch.cuda.synchronize()
    assert norm_err(got.cpu().numpy(), want.cpu().numpy()).max() <= TOL_F32
    # M = 0: the filter is the identity, s = e
    a0 = torch.zeros((2, 5000, 0), device=DEV)
    got0 = _noalloc(a0, e, None)
    torch.cuda.synchronize()
    assert torch.equal(got0, e)


def _largest_fitting_T(B, M):
    """Largest T whose scratch fits the fixed array (need(T) is searched
    by bisection; returns None if it is not monotone around the limit)."""
    lim = _lib.LP_NOALLOC_SCRATCH_BYTES
    lo, hi = 1, 1
    while _lib.lp_tv_workspace_bytes(B, hi, M) <= lim:
        hi *= 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if _lib.lp_tv_workspace_bytes(B, mid, M) <= lim:
            lo = mid
        else:
            hi = mid
    if _lib.lp_tv_workspace_bytes(B, lo, M) > lim or _lib.lp_tv_workspace_bytes(B, lo + 1, M) <= lim:
        return None
    return lo


def test_noalloc_size_boundary():
    """The largest problem whose scratch fits runs and matches the regular
    forward; one more sample is rejected with LP_ETOOBIG."""
    B, M = 1, 22
    T = _largest_fitting_T(B, M)
    if T is None:
        pytest.skip("scratch size not monotone in T around the limit")
    w = inputs.make("noallocmax", B, T, M, seed=24, gen="stable")
    a, e = (torch.tensor(x, device=DEV) for x in (w.a, w.e))
    want = ops.lp_tv_forward(a, e)
    got = _noalloc(a, e, None)
    torch.cuda.synchronize()
    assert norm_err(got.cpu().numpy(), want.cpu().numpy()).max() <= TOL_F32
    with pytest.raises(_lib.LPError) as ei:
        _lib.lp_tv_forward_noalloc_f32(B, T + 1, M, 16, 16, None, 16, None)
    assert ei.value.code == _lib.LP_ETOOBIG


def test_noalloc_allocates_no_device_memory():
    """Around a warmed-up call neither torch's allocator nor the device's
    free memory changes."""
    w = inputs.make("noallocmem", 3, 30000, 22, seed=25, gen="stable", with_zi=True)
    a, e, zi = (torch.tensor(x, device=DEV) for x in (w.a, w.e, w.zi))
    s = torch.empty((3, 30000), device=DEV)
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        _lib.lp_tv_forward_noalloc_f32(3, 30000, 22, a.data_ptr(), e.data_ptr(), zi.data_ptr(), s.data_ptr(), stream)

    call()
    torch.cuda.synchronize()
    alloc0, (free0, _) = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()
    call()
    torch.cuda.synchronize()
    alloc1, (free1, _) = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()
    assert alloc1 == alloc0 and free1 == free0, (alloc0, alloc1, free0, free1)
