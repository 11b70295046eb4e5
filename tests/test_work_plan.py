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
                            ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P,
                            P, P, P, P, ctypes.c_int64, ctypes.c_int64]
    return lib


def block_units(sizes, mixed, threads, ipt, src=None):
    """Source units of each target block, in the planner's block order."""
    unit = 2 if mixed else 1
    B = threads * ipt
    out = []
    for s, n in enumerate(sizes):
        sn = n if src is None else int(src[1][s])
        out += [(sn + unit - 1) // unit] * ((n + B - 1) // B)
    return out


def plan(wp, sizes, mixed, threads, ipt, jsplit, slots, cost=None, src=None):
    """cost: None or (chunk_units, [weights of each block's chunks])."""
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    padded = [(n + 1) // 2 * 2 if mixed else n for n in sizes]
    soff = np.concatenate([[0], np.cumsum(padded)]).astype(np.int64)
    n = int(offsets[-1])
    cw = cw_off = None
    if cost is not None:
        cw = np.ascontiguousarray(np.concatenate([np.asarray(w, np.int64) for w in cost[1]]), dtype=np.int64)
        cw_off = np.concatenate([[0], np.cumsum([len(w) for w in cost[1]])]).astype(np.int64)
    sb = None if src is None else np.ascontiguousarray(src[0], dtype=np.int64)
    sn = None if src is None else np.ascontiguousarray(src[1], dtype=np.int64)
    cap_b = sum((s + threads * ipt - 1) // (threads * ipt) for s in sizes)
    cap_p = slots * (jsplit + 1) + 1
    cap_s = cap_p + 2 * cap_b + 8
    blks = np.zeros((cap_b, 4), np.int32)
    segs = np.zeros((cap_s, 4), np.int32)
    seg_off = np.zeros(cap_p + 1, np.int32)
    nsl = np.zeros(n, np.uint16)
    meta = np.zeros(5, np.int64)
    rc = wp.wp_plan(len(sizes), offsets.ctypes.data, soff.ctypes.data, int(mixed), threads, ipt, jsplit, slots,
                    cap_b, cap_s, cap_p, blks.ctypes.data, segs.ctypes.data, seg_off.ctypes.data,
                    nsl.ctypes.data, meta.ctypes.data, None if sb is None else sb.ctypes.data,
                    None if sn is None else sn.ctypes.data, None if cw is None else cw.ctypes.data,
                    None if cw is None else cw_off.ctypes.data, 0 if cost is None else len(cost[1]),
                    1 if cost is None else int(cost[0]))
    assert rc == 0, rc
    nb_, ns_, grid, ndyn, rows = (int(x) for x in meta)
    return dict(offsets=offsets, soff=soff, blks=blks[:nb_], segs=segs[:ns_],
                seg_off=seg_off[:grid + ndyn + 1], nsl=nsl, grid=grid, n_dyn=ndyn, rows=rows,
                cost=cost, src=None if src is None else (sb, sn))


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
        if p["src"] is None:
            assert mine[0, 1] == soff[s] and mine[-1, 2] == soff[s + 1]
        else:  # explicit sources: [src_b, src_b + src_n rounded up to whole units)
            sb, sn = int(p["src"][0][s]), int(p["src"][1][s])
            assert mine[0, 1] == sb and mine[-1, 2] == sb + (sn + unit - 1) // unit * unit
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
    def src_units(s):
        if p["src"] is None:
            return (soff[s + 1] - soff[s]) // unit
        return (int(p["src"][1][s]) + unit - 1) // unit

    # per block: the weight of each of its source units
    if p["cost"] is None:
        uw = [np.full(src_units(sys_of_blk[b]), (blk[1] - blk[0] + 32 * ipt - 1) // (32 * ipt), np.int64)
              for b, blk in enumerate(blks)]
    else:  # chunk c of block b weighs cost[1][b][c] per unit
        cu = p["cost"][0]
        uw = [np.maximum(np.repeat(np.asarray(p["cost"][1][b], np.int64), cu)[:src_units(sys_of_blk[b])], 1)
              for b in range(len(blks))]
    upre = [np.concatenate([[0], np.cumsum(w)]) for w in uw]
    W = sum(int(x[-1]) for x in upre)
    Ws = W - W // 4 if p["n_dyn"] > 0 else W
    wmax = max(int(w.max()) for w in uw)
    for g in range(p["grid"]):
        share = 0
        for sg in segs[so[g]:so[g + 1]]:
            s0 = int(p["src"][0][sys_of_blk[sg[0]]]) if p["src"] is not None else int(soff[sys_of_blk[sg[0]]])
            u0, u1 = (int(sg[1]) - s0) // unit, (int(sg[2]) - s0) // unit
            share += int(upre[sg[0]][u1] - upre[sg[0]][u0])
        nseg = so[g + 1] - so[g]
        assert abs(share - Ws / p["grid"]) <= wmax * (nseg + 1), (g, share, Ws / p["grid"])
    # minimum piece length
    units = [src_units(sys_of_blk[b]) for b in range(len(blks))]
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


@pytest.mark.parametrize("mixed", [False, True])
def test_cost_weighted_plans(wp, mixed):
    """A cost model per block and chunk of sources (the mixed path's far/near
    estimate): the invariants hold and the static shares are equal in cost,
    so a costlier block gets more, shorter shares, and a costlier chunk
    shorter segments."""
    rng = np.random.default_rng(17 + mixed)
    for _ in range(60):
        n_sys = int(rng.integers(1, 4))
        sizes = [int(x) for x in rng.choice([31, 131, 700, 1531, 5003, 12000], n_sys)]
        threads, ipt = [(128, 1), (256, 1), (512, 1), (256, 2)][int(rng.integers(0, 4))]
        jsplit = int(rng.choice([0, 2, 8]))
        slots = int(rng.choice([7, 152, 304]))
        cu = int(rng.choice([1, 32, 96]))
        w = [rng.integers(96, 289, size=(u + cu - 1) // cu) for u in block_units(sizes, mixed, threads, ipt)]
        p = plan(wp, sizes, mixed, threads, ipt, jsplit, slots, cost=(cu, w))
        check(p, sizes, mixed, threads, ipt, jsplit, slots)
    # two blocks, one three times as costly: it gets about three times the shares
    sizes = [2048]
    units = block_units(sizes, True, 1024, 1)
    p = plan(wp, sizes, True, 1024, 1, 0, 152, cost=(32, [[100] * ((units[0] + 31) // 32), [300] * ((units[1] + 31) // 32)]))
    check(p, sizes, True, 1024, 1, 0, 152)
    per_blk = [int((p["segs"][:, 0] == b).sum()) for b in range(2)]
    assert 2.5 <= per_blk[1] / per_blk[0] <= 3.5, per_blk
    # one block whose second half of sources costs twice the first: segments
    # in the costly half are half as long
    sizes = [1024]
    units = block_units(sizes, True, 1024, 1)[0]  # 512 units, 16 chunks of 32
    p = plan(wp, sizes, True, 1024, 1, 0, 48, cost=(32, [[100] * 8 + [200] * 8]))
    check(p, sizes, True, 1024, 1, 0, 48)
    lens = (p["segs"][:, 2] - p["segs"][:, 1]) // 2
    first = lens[p["segs"][:, 2] <= units]  # segments inside the cheap half (units 0..256)
    last = lens[p["segs"][:, 1] >= units]   # inside the costly half
    assert len(first) and len(last)
    assert 1.6 <= first.mean() / last.mean() <= 2.4, (first.mean(), last.mean())


@pytest.mark.parametrize("mixed", [False, True])
def test_row_shard_plans(wp, mixed):
    """Row shards: one rank's targets (its block of bodies) against every
    source entry of the stage (world chunks of C entries): each block's
    segments tile the whole source range, and the shares stay balanced."""
    for n, world, rank in ((1001, 2, 1), (10425, 3, 0), (10425, 3, 2), (5, 4, 1)):
        c = ((n + world - 1) // world + 1) // 2 * 2
        b, e = min(rank * c, n), min(rank * c + c, n)
        if e <= b:
            continue
        p = plan(wp, [e - b], mixed, 256, 1, 0, 152, src=([0], [world * c]))
        check(p, [e - b], mixed, 256, 1, 0, 152)
