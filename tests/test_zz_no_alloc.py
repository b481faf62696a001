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
