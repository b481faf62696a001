"""Failure detection on the GPU without a fault: the kernels' bounded waits.

lp_tv_selftest_wait runs one warp through the library's own wait
primitives on a condition nothing satisfies (an mbarrier waiting for
bulk-copy bytes never sent, a progress counter nothing increments).  The
wait must give up within its limit, record its status in the device status
word (1: copy wait, 2: scan counter wait), return, and leave the context
usable: a normal call afterwards is correct and reports no error.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2406_05128_gb300 import _lib, inputs, ops  # noqa: E402
from tests.helpers import TOL_F32, assert_close  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


@pytest.mark.parametrize("which", [1, 2])
def test_bounded_wait_gives_up_reports_and_context_survives(which):
    lib = _lib.load()
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status(reset=True) in (0, 1, 2)
    assert _lib.lp_tv_device_status() == 0
    t0 = time.perf_counter()
    assert lib.lp_tv_selftest_wait(which, torch.cuda.current_stream().cuda_stream) == 0
    status = _lib.lp_tv_device_status(reset=True)  # synchronises
    dt = time.perf_counter() - t0
    assert status == which
    assert dt < 10.0, dt
    # the context is usable: a normal forward + adjoint, against the oracle
    w = inputs.make("fail", 2, 3000, 22, seed=4, gen="stable", with_zi=True)
    a, e, gs, zi = (torch.tensor(x, device="cuda") for x in (w.a, w.e, w.gs, w.zi))
    s = ops.lp_tv_forward(a, e, zi)
    ge, ga, _ = ops.lp_tv_backward(gs, a, s, zi)
    torch.cuda.synchronize()
    assert _lib.lp_tv_device_status() == 0
    rs, rge, rga, _ = O.forward_backward(w.a, w.e, w.gs, w.zi)
    assert_close("s", s.cpu().numpy(), rs, TOL_F32)
    assert_close("ge", ge.cpu().numpy(), rge, TOL_F32)
    print(f"wait {which} gave up after {dt:.3f} s")
