"""lp_tv_check_finite_*: the non-finite check agrees with numpy.isfinite on
every shape of input the kernel splits differently (a misaligned head, the
16-byte vectors, a ragged tail), for a single bad element anywhere, and on a
real forward output that overflowed (the literal generator at M=22)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2406_05128_gb300 import _lib, inputs, ops  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    _lib.load()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 31, 1000, (1 << 20) + 3])
@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_single_bad_element_anywhere(dtype, n, offset):
    base = torch.randn(n + offset, dtype=dtype, device=DEV)
    x = base[offset:]  # misaligned starts exercise the scalar head
    assert ops.all_finite(x)
    positions = sorted({0, n // 2, n - 1, max(0, n - 2), min(n - 1, 3)})
    for pos in positions:
        for bad in (float("nan"), float("inf"), float("-inf")):
            y = x.clone() if offset == 0 else base.clone()[offset:]
            y[pos] = bad
            assert not ops.all_finite(y), (n, offset, pos, bad)


def test_empty_and_large_values():
    assert _lib.lp_tv_check_finite(_lib.LP_DTYPE_F32, torch.empty(0, device=DEV).data_ptr(), 0,
                                   torch.cuda.current_stream().cuda_stream)
    x = torch.full((4096,), 3.0e38, device=DEV)  # large but finite
    assert ops.all_finite(x)
    x[4095] = float("inf")
    assert not ops.all_finite(x)


def test_forward_output_matches_numpy():
    """A forward on the literal |k| <= 0.95 generator at M=22: whatever the
    draw does, the check agrees with numpy on the output; the stable
    generator's output is finite."""
    for gen in ("literal", "stable"):
        w = inputs.make("chk", 4, 48000, 22, seed=2, gen=gen, excitation="pulse")
        a, e = torch.tensor(w.a, device=DEV), torch.tensor(w.e, device=DEV)
        s = ops.lp_tv_forward(a, e)
        torch.cuda.synchronize()
        expect = bool(np.isfinite(s.cpu().numpy()).all())
        assert ops.all_finite(s) == expect
        if gen == "stable":
            assert expect
        assert ops.all_finite(a) and ops.all_finite(e)


def test_lp_filter_check_raises_on_overflow_and_passes_when_stable():
    """ops.lp_filter(check=True): a filter with a pole outside the unit
    circle overflows and raises; a stable one runs forward and backward."""
    T, M = 4000, 2
    a = torch.zeros((1, T, M), device=DEV)
    a[..., 0] = -2.5  # s(t) = e(t) + 2.5 s(t-1): grows as 2.5^t
    e = torch.ones((1, T), device=DEV)
    with pytest.raises(FloatingPointError):
        ops.lp_filter(a, e, check=True)
    w = inputs.make("chk2", 2, 3000, 16, seed=4, gen="stable")
    a2 = torch.tensor(w.a, device=DEV, requires_grad=True)
    e2 = torch.tensor(w.e, device=DEV, requires_grad=True)
    s = ops.lp_filter(a2, e2, check=True)
    s.sum().backward()
    assert ops.all_finite(a2.grad) and ops.all_finite(e2.grad)
