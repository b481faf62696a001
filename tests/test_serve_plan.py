"""The serving loop's planner (host logic, no GPU): the same C++ planner the
engine runs, driven by a step simulation (libtvlp_plan.so).

Checked on random arrival streams:
- every request's rows are covered exactly once, in order, by its blocks;
  synthesis blocks hold at most block_rows rows, adaptation requests run
  whole in one block;
- continuing blocks open the next iteration, in the previous order, and
  start from a carried state; a block is carried exactly when it is not its
  request's first;
- admission is FIFO: requests start in arrival order;
- every call is packed back to back from row 0 with even (16-byte aligned)
  signal starts; calls stay within max_signals and the iteration within
  max_iter_rows;
- iteration regions fit the ring and regions alive at the same time never
  overlap (the HBM budget is respected).
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2406_05128_gb300 import build


@pytest.fixture(scope="module")
def plan():
    lib = ctypes.CDLL(build.build_plan())
    i32, i64, u64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
    lib.lp_plan_simulate.argtypes = [i32, i64, i32, i64, u64, i32, i32, i32, vp, vp, vp, i64, vp, i64, vp, vp, vp]
    lib.lp_plan_simulate.restype = i32
    lib.lp_plan_layout.argtypes = [i32, i64, i32, i64, i32, i32, i64, i64, vp]
    lib.lp_plan_layout.restype = i32
    lib.lp_plan_max_region_bytes.argtypes = [i32, i64, i32, i64]
    lib.lp_plan_max_region_bytes.restype = u64
    return lib


def simulate(lib, T, kind, arrive, *, M=22, block_rows=4096, max_signals=8, max_iter_rows=1 << 16,
             ring_bytes=None, lag=3, hop=0):
    T = np.ascontiguousarray(T, dtype=np.int64)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    arrive = np.ascontiguousarray(arrive, dtype=np.int64)
    if ring_bytes is None:
        ring_bytes = 2 * lib.lp_plan_max_region_bytes(M, block_rows, max_signals, max_iter_rows)
    cap = int(4 * (T.sum() // max(block_rows, 1) + len(T)) + 64)
    blocks = np.zeros((cap, 9), np.int64)
    iters = np.zeros((cap, 5), np.uint64)
    nb, ni = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.lp_plan_simulate(M, block_rows, max_signals, max_iter_rows, ring_bytes, hop, lag, len(T), T.ctypes.data,
                              kind.ctypes.data, arrive.ctypes.data, cap, blocks.ctypes.data, cap,
                              iters.ctypes.data, ctypes.byref(nb), ctypes.byref(ni))
    return rc, blocks[:nb.value], iters[:ni.value], ring_bytes


def layout_bytes(lib, M, rf, nf, ra, na, nc, frames_f=-1, frames_a=0):
    out = np.zeros(15, np.uint64)
    assert lib.lp_plan_layout(M, rf, nf, ra, na, nc, frames_f, frames_a, out.ctypes.data) == 0
    return out


def check(lib, T, kind, blocks, iters, ring_bytes, *, M, block_rows, max_signals, max_iter_rows, hop=0):
    n = len(T)
    # coverage, order, block sizes, carried flags
    per_req = {k: [] for k in range(n)}
    for it, rq, row0, rows, pos, call, carried, last, fpos in blocks:
        per_req[int(rq)].append((int(it), int(row0), int(rows), int(call), int(carried), int(last)))
    first_iter = []
    for k in range(n):
        bl = per_req[k]
        assert bl, f"request {k} never planned"
        its = [b[0] for b in bl]
        assert its == sorted(its) and len(set(its)) == len(its)
        row = 0
        for j, (it, row0, rows, call, carried, last) in enumerate(bl):
            assert row0 == row
            row += rows
            assert call == kind[k]
            assert carried == (1 if j > 0 else 0)
            assert last == (1 if j == len(bl) - 1 else 0)
            if kind[k] == 1:
                assert rows == T[k] and len(bl) == 1
            elif block_rows > 0:
                assert rows <= block_rows
                if not last:
                    assert rows == block_rows
            # consecutive blocks of a request run in consecutive iterations
            if j > 0:
                assert it == bl[j - 1][0] + 1
        assert row == T[k]
        first_iter.append(bl[0][0])
    # FIFO admission
    assert first_iter == sorted(first_iter)
    # per iteration: packing, limits, continuing first
    prev_cont = []
    for i in range(len(iters)):
        b = blocks[blocks[:, 0] == i]
        fw, ad = b[b[:, 5] == 0], b[b[:, 5] == 1]
        for call in (fw, ad):
            assert len(call) <= max_signals
            pos = 0
            for r in call:
                assert r[4] == pos and pos % 2 == 0
                pos += int(r[3]) + int(r[3]) % 2
        rows_f = int(sum(int(r[3]) + int(r[3]) % 2 for r in fw))
        rows_a = int(sum(int(r[3]) + int(r[3]) % 2 for r in ad))
        assert rows_f + rows_a <= max_iter_rows
        ncar = int(fw[:, 6].sum()) if len(fw) else 0
        assert list(fw[:ncar, 1]) == prev_cont
        assert np.all(fw[ncar:, 6] == 0) if len(fw) else True
        prev_cont = [int(r[1]) for r in fw if r[7] == 0]
        nc = len(prev_cont)
        frames_f, frames_a = -1, 0
        if hop > 0:
            # blocks start on frame anchors; frame rows packed back to back in
            # each call
            def packed_frames(call):
                fpos = 0
                for r in call:
                    assert r[2] % hop == 0 and r[8] == fpos
                    fpos += -(-(int(r[3]) + int(r[3]) % 2) // hop) + 1
                return fpos
            frames_f, frames_a = packed_frames(fw), packed_frames(ad)
        lay = layout_bytes(lib, M, rows_f, len(fw), rows_a, len(ad), nc, frames_f, frames_a)
        assert int(iters[i, 3]) == int(lay[14])
    # ring: in bounds, no overlap between regions alive at the same time
    for i in range(len(iters)):
        off, nbytes = int(iters[i, 2]), int(iters[i, 3])
        assert off % 256 == 0 and off + nbytes <= ring_bytes
        assert int(iters[i, 4]) <= ring_bytes
    for i in range(len(iters)):
        for j in range(i + 1, len(iters)):
            si, ei = int(iters[i, 0]), int(iters[i, 1])
            sj = int(iters[j, 0])
            if sj >= ei:  # i completed before j was planned
                continue
            a0, a1 = int(iters[i, 2]), int(iters[i, 2]) + int(iters[i, 3])
            b0, b1 = int(iters[j, 2]), int(iters[j, 2]) + int(iters[j, 3])
            assert a1 <= b0 or b1 <= a0, (i, j)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_streams(plan, seed):
    rng = np.random.default_rng(seed)
    n = 60
    T = rng.integers(0, 20000, size=n)
    T[::13] = rng.integers(0, 3, size=T[::13].shape)  # empty and one-sample requests
    kind = (rng.random(n) < 0.2).astype(np.int32)
    arrive = np.sort(rng.integers(0, 80, size=n))
    cfg = dict(M=22, block_rows=4096, max_signals=6, max_iter_rows=1 << 15)
    rc, blocks, iters, ring = simulate(plan, T, kind, arrive, **cfg)
    assert rc == 0
    check(plan, T, kind, blocks, iters, ring, **cfg)
    # the stream exercised what the checks are about
    assert blocks[:, 6].sum() > 0                       # carried states
    assert np.bincount(blocks[:, 0]).max() > 1          # batched iterations
    assert np.any((blocks[:, 5] == 0) & np.isin(blocks[:, 0], blocks[blocks[:, 5] == 1, 0]))  # both calls


def test_tight_budget_still_serves_everything(plan):
    """A ring that holds about one largest iteration: requests wait for
    memory, none is lost or reordered."""
    rng = np.random.default_rng(7)
    n = 40
    T = rng.integers(1000, 30000, size=n)
    kind = (rng.random(n) < 0.3).astype(np.int32)
    arrive = np.zeros(n, np.int64)
    cfg = dict(M=16, block_rows=2048, max_signals=4, max_iter_rows=32768)
    ring = int(plan.lp_plan_max_region_bytes(16, 2048, 4, 32768)) + 4096
    rc, blocks, iters, ring = simulate(plan, T, kind, arrive, ring_bytes=ring, **cfg)
    assert rc == 0
    check(plan, T, kind, blocks, iters, ring, **cfg)
    assert int(iters[:, 4].max()) <= ring
    offs = iters[:, 2].astype(np.int64)
    assert np.any(np.diff(offs) < 0)  # the ring wrapped around


def test_whole_requests_without_blocks(plan):
    rng = np.random.default_rng(9)
    T = rng.integers(0, 9000, size=25)
    kind = np.zeros(25, np.int32)
    arrive = np.arange(25) // 3
    cfg = dict(M=30, block_rows=0, max_signals=5, max_iter_rows=20000)
    rc, blocks, iters, ring = simulate(plan, T, kind, arrive, **cfg)
    assert rc == 0
    check(plan, T, kind, blocks, iters, ring, **cfg)
    assert np.all(blocks[:, 6] == 0) and np.all(blocks[:, 7] == 1)


def test_long_request_does_not_hold_back_short_ones(plan):
    """A 20-block utterance arrives first; short requests that arrive after
    it start within one iteration of their arrival, not after it ends."""
    T = np.array([20 * 4096] + [3000] * 10)
    kind = np.zeros(11, np.int32)
    arrive = np.array([0] + list(range(2, 12)))
    cfg = dict(M=22, block_rows=4096, max_signals=8, max_iter_rows=1 << 16)
    rc, blocks, iters, ring = simulate(plan, T, kind, arrive, lag=1, **cfg)
    assert rc == 0
    check(plan, T, kind, blocks, iters, ring, **cfg)
    step_of = {int(i): int(iters[i, 0]) for i in range(len(iters))}
    for k in range(1, 11):
        it = int(blocks[blocks[:, 1] == k][0, 0])
        assert step_of[it] - arrive[k] <= 1
    last_long = int(blocks[(blocks[:, 1] == 0) & (blocks[:, 7] == 1)][0, 0])
    assert all(int(blocks[blocks[:, 1] == k][0, 0]) < last_long for k in range(1, 11))


def test_oversized_requests_rejected(plan):
    T = np.array([70000])
    rc, *_ = simulate(plan, T, np.array([1], np.int32), np.array([0]), max_iter_rows=1 << 16)
    assert rc == -1  # an adaptation request runs whole: larger than an iteration
    rc, *_ = simulate(plan, T, np.array([0], np.int32), np.array([0]), max_iter_rows=1 << 16)
    assert rc == 0  # a synthesis request is cut into blocks


def test_layout_is_aligned_and_disjoint(plan):
    lay = layout_bytes(plan, 22, 1002, 3, 998, 2, 1)
    # frames mode: the synthesis call holds 12 frame rows, and a frame-offset
    # table sits between the row offsets and the continuing indexes
    lf = layout_bytes(plan, 22, 1002, 3, 998, 2, 1, 12, 11)
    assert int(lf[1]) - int(lf[0]) >= 12 * 88 and int(lf[1]) < int(lay[1])
    assert int(lf[4]) - int(lf[3]) >= 11 * 88 and int(lf[4]) - int(lf[3]) < 998 * 88  # a_a holds 11 frames
    assert int(lf[12]) - int(lf[11]) == 3 * 8 + 3 * 8 + 2 * 8
    starts = [int(x) for x in lay[:9]] + [int(lay[9])]
    sizes = [1002 * 88, 1002 * 4, 1002 * 4, 998 * 88, 998 * 4, 998 * 4, 998 * 4, 998 * 4, 998 * 88]
    for s in starts:
        assert s % 256 == 0
    for (s0, n0), s1 in zip(zip(starts[:9], sizes), starts[1:]):
        assert s0 + n0 <= s1
    # tables: off_f [4] int64, off_a [3] int64, cont [1] int32
    assert int(lay[11]) - int(lay[10]) == 4 * 8 and int(lay[12]) - int(lay[11]) == 3 * 8
    assert int(lay[13]) == 4 * 8 + 3 * 8 + 4 and int(lay[14]) >= int(lay[12]) + 4


def test_frames_server_plan(plan):
    """hop > 0: blocks start on frame anchors and both calls carry their
    frame rows packed back to back, adaptation requests included."""
    rng = np.random.default_rng(11)
    n = 40
    T = rng.integers(0, 20000, size=n)
    kind = (rng.random(n) < 0.25).astype(np.int32)
    arrive = np.sort(rng.integers(0, 50, size=n))
    cfg = dict(M=22, block_rows=4800, max_signals=6, max_iter_rows=1 << 15, hop=120)
    rc, blocks, iters, ring = simulate(plan, T, kind, arrive, **cfg)
    assert rc == 0
    check(plan, T, kind, blocks, iters, ring, **cfg)
    assert blocks[:, 6].sum() > 0 and (blocks[:, 5] == 1).sum() > 0
