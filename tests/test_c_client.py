"""The C ABI from plain C: tests/c_client/tvlp_client.c (no Python, no
PyTorch) is compiled with gcc against include/tvlp.h and linked with
libtvlp.so and the CUDA runtime.  On the CPU it must compile and link; on
the GPU its forward + adjoint must match the FP64 oracle."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "tvlp_client.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build_client(tmp_path):
    from paper_2406_05128_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "tvlp_client")
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           SRC, "-o", exe, "-L", os.path.dirname(lib), "-ltvlp", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.dirname(lib), "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


@pytest.mark.skipif(shutil.which("gcc") is None or not os.path.exists(os.path.join(CUDA, "include")),
                    reason="gcc or the CUDA headers are missing")
def test_c_client_compiles_and_links(tmp_path):
    exe = _build_client(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_client_matches_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from paper_2406_05128_gb300 import inputs
    from tests.helpers import TOL_F32, assert_close
    exe = _build_client(tmp_path)
    B, T, M = 3, 4000, 22
    w = inputs.make("cclient", B, T, M, seed=17, gen="stable", with_zi=True)
    din, dout = tmp_path / "in", tmp_path / "out"
    din.mkdir()
    dout.mkdir()
    for name, x in (("a", w.a), ("e", w.e), ("gs", w.gs), ("zi", w.zi)):
        np.ascontiguousarray(x, np.float32).tofile(din / f"{name}.bin")
    res = subprocess.run([exe, str(B), str(T), str(M), str(din), str(dout)], capture_output=True, text=True,
                         timeout=120)
    assert res.returncode == 0, res.stderr + res.stdout
    got = {n: np.fromfile(dout / f"{n}.bin", np.float32) for n in ("s", "ge", "ga", "gzi")}
    rs, rge, rga, rgzi = O.forward_backward(w.a, w.e, w.gs, w.zi)
    assert_close("s", got["s"].reshape(B, T), rs, TOL_F32)
    assert_close("ge", got["ge"].reshape(B, T), rge, TOL_F32)
    assert_close("ga", got["ga"].reshape(B, T, M), rga, TOL_F32)
    d = np.abs(got["gzi"].reshape(B, M) - rgzi).max(axis=1) / np.abs(rge).max(axis=1)
    assert d.max() <= TOL_F32
