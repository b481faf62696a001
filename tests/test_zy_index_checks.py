"""The checked build: index checks inside the kernels (TVLP_CHECK_BOUNDS).

A library compiled with TVLP_CHECK_BOUNDS checks, on the device, every index
that comes from a table or a list the kernels build themselves: a chunk's
signal in a varlen batch, a scan item's signal and group, a group's chunks,
the chain's groups, the correction list's slots and entries.  A failed check
records 16 + its location in the status word and skips the work it guards,
so it never faults.  This test builds that library into its own folder and
runs a selection of the parity tests against it in a fresh process: those
tests assert that the status word stays 0 after every call and that the
results meet the oracle.  The selection covers ragged tails, T < M, padded
orders, the chain blocks and the grids without room for them, resonant
signals whose correction lists chunks, varlen batches with empty signals,
mixed orders, generated coefficients and checkpoints.
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = [
    "tests/test_gpu_parity.py::test_parity_f32",
    "tests/test_gpu_parity.py::test_literal_generator_k08_ill_conditioned",
    "tests/test_gpu_parity.py::test_scan_without_room_for_chain_blocks",
    "tests/test_gpu_parity.py::test_scan_chain_longer_than_chain_ring",
    "tests/test_gpu_parity.py::test_degenerate_sizes",
    "tests/test_gpu_varlen.py::test_varlen_matches_oracle",
    "tests/test_gpu_varlen.py::test_varlen_alone_equals_in_the_mix_resonant",
    "tests/test_gpu_varlen.py::test_mixed_orders_match_oracle",
    "tests/test_gpu_varlen.py::test_mixed_resonant_signals",
    "tests/test_gpu_frames.py::test_frames_match_oracle",
    "tests/test_gpu_frames.py::test_frames_resonant_with_and_without_row_cache",
    "tests/test_gpu_checkpoint.py::test_recompute_bitwise_with_defect_correction",
    "tests/test_gpu_fused_grad.py::test_resonant_fused_equals_separate",
]


def test_checked_build_runs_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_05128_gb300 import build
    lib = build.build(checks=True)
    env = dict(os.environ, TVLP_LIBRARY=lib)
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                          *SELECTION], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((res.stdout + res.stderr).splitlines()[-30:])
    assert res.returncode == 0, tail
    assert " passed" in res.stdout, tail
