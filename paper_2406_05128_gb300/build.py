"""Build the CUDA library libtvlp.so for sm_103a, in-tree.

Each (scalar type, padded order) instantiation is its own translation unit,
compiled in parallel with nvcc, then linked with the C ABI and the serving
engine into one shared library: paper_2406_05128_gb300/_build/libtvlp.so.
The serving loop's planner is also built alone with the host compiler
(libtvlp_plan.so, no CUDA) for its CPU simulation.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libtvlp.so")
PLAN_LIB = os.path.join(BUILD, "libtvlp_plan.so")
# the checked build (index checks in the kernels, TVLP_CHECK_BOUNDS): a
# library of its own for tests, never the one the package loads
BUILD_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libtvlp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]

F32_ORDERS = (2, 4, 8, 12, 16, 22, 30, 32)
F64_ORDERS = (2, 4, 8, 12, 16)


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtvlp")
    return path


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]


def _units(out=BUILD):
    units = []
    for scalar, orders in (("float", F32_ORDERS), ("double", F64_ORDERS)):
        for mp in orders:
            obj = os.path.join(out, f"inst_{scalar}_{mp}.o")
            units.append((os.path.join(CSRC, "tvlp_inst.cu"), obj,
                          [f"-DTVLP_SCALAR={scalar}", f"-DTVLP_MP={mp}"]))
    for name in ("tvlp_api", "tvlp_noalloc", "tvlp_serve", "tvlp_selftest", "tvlp_check", "tvlp_framewise"):
        units.append((os.path.join(CSRC, name + ".cu"), os.path.join(out, name + ".o"), []))
    # mixed orders: the host side, and the fused kernels in parallel parts
    units.append((os.path.join(CSRC, "tvlp_mixed.cu"), os.path.join(out, "tvlp_mixed.o"), []))
    units.append((os.path.join(CSRC, "tvlp_mixed_k1.cu"), os.path.join(out, "tvlp_mixed_k1.o"), []))
    for name in ("tvlp_mixed_rec", "tvlp_mixed_scan"):
        for part in (0, 1):
            units.append((os.path.join(CSRC, name + ".cu"), os.path.join(out, f"{name}_{part}.o"),
                          [f"-DTVLP_MIX_PART={part}"]))
    return units


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(unit, verbose: bool, ptxas_v: bool, checks: bool = False):
    src, obj, defs = unit
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *defs, *(["-DTVLP_CHECK_BOUNDS"] if checks else []), "-c", src, "-o", obj]
    if ptxas_v:
        cmd += ["-Xptxas", "-v"]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{res.stderr}")
    return res.stderr


def build_plan(force: bool = False) -> str:
    """The planner simulation library (host compiler only)."""
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(CSRC, "serve_sim.cpp")
    deps = [src, os.path.join(CSRC, "serve_plan.h")]
    if force or _stale(PLAN_LIB, deps):
        cxx = shutil.which("g++") or shutil.which("c++")
        if cxx is None:
            raise RuntimeError("no host C++ compiler found for libtvlp_plan.so")
        tmp = PLAN_LIB + f".tmp{os.getpid()}"
        cmd = [cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, src, "-o", tmp]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"host build of libtvlp_plan.so failed:\n{res.stderr}")
        os.replace(tmp, PLAN_LIB)
    return PLAN_LIB


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, jobs: int | None = None,
          checks: bool = False) -> str:
    """Compile every instantiation (in parallel) and link libtvlp.so; with
    checks=True the checked build (index checks in the kernels) into its
    own folder."""
    out, lib = (BUILD_CHECK, LIB_CHECK) if checks else (BUILD, LIB)
    os.makedirs(out, exist_ok=True)
    deps = _sources()
    units = _units(out)
    todo = [u for u in units if force or ptxas_v or _stale(u[1], deps)]
    if todo:
        jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with ThreadPoolExecutor(jobs) as ex:
            logs = list(ex.map(lambda u: _compile(u, verbose, ptxas_v, checks), todo))
        if ptxas_v:
            for u, log in zip(todo, logs):
                print(f"== {os.path.basename(u[1])}\n{log}")
    objs = [u[1] for u in units]
    if force or todo or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr}")
        os.replace(tmp, lib)
    if not checks:
        build_plan(force)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_v="--ptxas" in sys.argv))
