"""The host work planner of the force and VJP launches (csrc/work_plan.h),
built with g++ through tests/work_plan_shim.cpp and checked on the CPU.

A wrong plan would drop or double-count interactions of Eq. 1, or break the
fixed summation order, on every launch.  For seeded random systems, tiles and
SM counts these tests check:
- each system's targets are cut into contiguous blocks of balanced size;
- each block's segments tile the system's stage range exactly, in slot order
  (slot = the partial row and the place in the sum), at even boundaries on
  the mixed path (its stage holds source pairs);
- every segment is in exactly one piece; the static shares are balanced;
- each body's row count is its block's segment count;
- small systems get fewer, longer pieces (at least c * sqrt(U) units).
"""
import ctypes
import math
import shutil
import subprocess

import numpy as np
import pytest

import os

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_15079_gb300", "csrc")


@pytest.fixture(scope="module")
def wp(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("wp") / "libwp.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "work_plan_shim.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.wp_plan.restype = ctypes.c_int
    lib.wp_plan.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P]
    return lib


def plan(wp, sizes, mixed, threads, ipt, jsplit, slots):
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    padded = [(n + 1) // 2 * 2 if mixed else n for n in sizes]
    soff = np.concatenate([[0], np.cumsum(padded)]).astype(np.int64)
    n = int(offsets[-1])
    cap_b = sum((s + threads * ipt - 1) // (threads * ipt) for s in sizes)
    cap_p = slots * (jsplit + 1) + 1
    cap_s = cap_p + cap_b + 8
    blks = np.zeros((cap_b, 4), np.int32)
    segs = np.zeros((cap_s, 4), np.int32)
    seg_off = np.zeros(cap_p + 1, np.int32)
    nsl = np.zeros(n, np.uint16)
    meta = np.zeros(5, np.int64)
    rc = wp.wp_plan(len(sizes), offsets.ctypes.data, soff.ctypes.data, int(mixed), threads, ipt, jsplit, slots,
                    cap_b, cap_s, cap_p, blks.ctypes.data, segs.ctypes.data, seg_off.ctypes.data,
                    nsl.ctypes.data, meta.ctypes.data)
    assert rc == 0, rc
    nb_, ns_, grid, ndyn, rows = (int(x) for x in meta)
    return dict(offsets=offsets, soff=soff, blks=blks[:nb_], segs=segs[:ns_],
                seg_off=seg_off[:grid + ndyn + 1], nsl=nsl, grid=grid, n_dyn=ndyn, rows=rows)


def check(p, sizes, mixed, threads, ipt, jsplit, slots):
    unit = 2 if mixed else 1
    B = threads * ipt
    offsets, soff, blks, segs = p["offsets"], p["soff"], p["blks"], p["segs"]
    # blocks: per system contiguous, balanced, within B, stage index q0
    sys_of_blk = []
    k = 0
    for s, n in enumerate(sizes):
        nb_s = (n + B - 1) // B
        mine = blks[k:k + nb_s]
        k += nb_s
        assert mine[0, 0] == offsets[s] and mine[-1, 1] == offsets[s + 1]
        assert np.all(mine[1:, 0] == mine[:-1, 1])
        lens = mine[:, 1] - mine[:, 0]
        assert lens.max() <= B and lens.max() - lens.min() <= 1 and lens.min() >= 1
        assert np.all(mine[:, 2] == soff[s] + (mine[:, 0] - offsets[s]))
        sys_of_blk += [s] * nb_s
    assert k == len(blks)
    # segments of each block tile [soff[s], soff[s+1]) in slot order
    for b, blk in enumerate(blks):
        s = sys_of_blk[b]
        mine = segs[segs[:, 0] == b]
        assert len(mine) == blk[3] >= 1
        mine = mine[np.argsort(mine[:, 3])]
        assert np.array_equal(mine[:, 3], np.arange(len(mine)))
        assert mine[0, 1] == soff[s] and mine[-1, 2] == soff[s + 1]
        assert np.all(mine[1:, 1] == mine[:-1, 2]) and np.all(mine[:, 2] > mine[:, 1])
        if mixed:
            assert np.all(mine[:, 1] % 2 == 0) and np.all(mine[:, 2] % 2 == 0)
    # pieces: seg_off partitions the segment list; slots rise with the piece index
    so = p["seg_off"]
    assert so[0] == 0 and so[-1] == len(segs) and np.all(np.diff(so) >= 0)
    assert len(so) == p["grid"] + p["n_dyn"] + 1
    assert 1 <= p["grid"] <= slots and p["n_dyn"] <= jsplit * p["grid"]
    last_slot = {}
    for g in range(len(so) - 1):
        for sg in segs[so[g]:so[g + 1]]:
            assert sg[3] == last_slot.get(sg[0], -1) + 1
            last_slot[sg[0]] = sg[3]
    # rows per body
    for blk in blks:
        assert np.all(p["nsl"][blk[0]:blk[1]] == blk[3])
    assert p["rows"] == blks[:, 3].max()
    # static shares: equal weighted length up to one unit's rounding per segment
    w = [(min(threads, blk[1] - blk[0]) + 31) // 32 for blk in blks]
    W = sum(((soff[sys_of_blk[b] + 1] - soff[sys_of_blk[b]]) // unit) * w[b] for b in range(len(blks)))
    Ws = W - W // 4 if p["n_dyn"] > 0 else W
    wmax = max(w)
    for g in range(p["grid"]):
        share = sum((sg[2] - sg[1]) // unit * w[sg[0]] for sg in segs[so[g]:so[g + 1]])
        nseg = so[g + 1] - so[g]
        assert abs(share - Ws / p["grid"]) <= wmax * (nseg + 1), (g, share, Ws / p["grid"])
    # minimum piece length
    units = [(soff[sys_of_blk[b] + 1] - soff[sys_of_blk[b]]) // unit for b in range(len(blks))]
    umax = max(units)
    c = 0.5 if mixed else (1.0 if umax < 800 else 2.0 if umax < 2000 else 3.0)
    umin = max(1, math.ceil(c * math.sqrt(umax)))
    if p["grid"] < slots:  # the rule bound: shares are at least umin units on average
        assert sum(units) / p["grid"] >= umin




@pytest.mark.parametrize("mixed", [False, True])
def test_random_plans(wp, mixed):
    rng = np.random.default_rng(7 + mixed)
    for _ in range(120):
        n_sys = int(rng.integers(1, 6))
        sizes = [int(x) for x in rng.choice([1, 2, 3, 31, 64, 131, 700, 1531, 5003, 12000], n_sys)]
        threads, ipt = [(64, 1), (128, 1), (256, 1), (512, 1), (1024, 1), (256, 2), (384, 2), (128, 4)][
            int(rng.integers(0, 8))]
        jsplit = int(rng.choice([0, 0, 1, 4]))
        slots = int(rng.choice([1, 7, 152, 304, 456, 608]))
        p = plan(wp, sizes, mixed, threads, ipt, jsplit, slots)
        check(p, sizes, mixed, threads, ipt, jsplit, slots)


def test_benchmark_and_small_system_plans(wp):
    # the 10,425-body mixed benchmark (512 x 1, 2 CTAs on 152 SMs): every slot used
    p = plan(wp, [10425], True, 512, 1, 0, 304)
    check(p, [10425], True, 512, 1, 0, 304)
    assert p["grid"] == 304 and p["n_dyn"] == 0
    # FP64 at 131 bodies (128 x 1, 3 CTAs on 152 SMs): short pieces are merged,
    # 131 rows per body would otherwise be summed in FP64
    p = plan(wp, [131], False, 128, 1, 0, 456)
    check(p, [131], False, 128, 1, 0, 456)
    assert p["rows"] <= 12 and p["grid"] == 262 // 12
    # one body, one system of one block
    p = plan(wp, [1], True, 512, 1, 4, 304)
    check(p, [1], True, 512, 1, 4, 304)
    assert p["grid"] == 1 and p["rows"] == 1
