"""The schedules of the pair-once kernels, emulated on the CPU.

The kernels cannot run here, but their decompositions are plain index
arithmetic, restated below from the kernels' own descriptions (csrc/sym.cu,
csrc/sym_mixed.cu) and checked for the properties the results rely on:

* wide FP64 blocks (force_sym_wide_kernel): T tiles of 32 bodies per block,
  four warps per CTA; in round r warp w holds tile p = 4 r + w of block I
  and in phase t rotates tile q = (p + t) mod T of block J past it; a
  diagonal item takes q > p in full and q == p as the half rotation
  (offsets 1..16 for the target, 1..15 for the reaction).
* mixed blocks (force_msym_kernel): T tiles per block, W = T / 4 warps;
  warp p holds entries 128 p + 32 a + l (slot a, lane l); in phase t it
  takes chunk c = (2 p + t) mod (T / 2), and at step k lane l takes the
  entries 64 c + 2 m + h (h = 0, 1) of pair block m = (l + k) mod 32; a
  diagonal item counts a pair only if the target's entry precedes the
  source's, and skips chunks wholly below the warp's entries.

Checked: within a phase no two warps touch the same J tile (chunk), so the
shared reaction sums need no atomics and take their terms in phase order;
an off-diagonal item meets every (target, source) pair exactly once; a
diagonal item counts every unordered pair of distinct entries exactly once,
for the target and for the reaction, and never an entry with itself; the
reaction sums of a pair block sit, after 16 steps, in the lane the kernel
folds them from; and the item list gives every body exactly one value in
each of its system's rows 0 .. blocks - 1 (ragged and exact block counts),
which the per-body kernel adds in order.  A planted error in the schedule
fails the checks.
"""
from collections import Counter

import pytest


def wide_fp64_item(T, diag, warps=4):
    """(phase-exclusivity ok, Counter of (target, source, side)) for one item
    of the wide FP64 kernel; bodies are local indices 0 .. 32 T - 1 of each
    block (the same block when diag)."""
    seen = Counter()
    exclusive = True
    for r in range(0, T, warps):
        for t in range(T):
            owners = [(r + w + t) % T for w in range(warps)]
            exclusive &= len(set(owners)) == warps
            for w in range(warps):
                p = r + w
                q = (p + t) % T
                if diag and q < p:
                    continue
                for lane in range(32):
                    tgt = 32 * p + lane
                    if diag and q == p:
                        for k in range(1, 17):
                            src = 32 * q + (lane + k) % 32
                            seen[(tgt, src, "target")] += 1
                            if k < 16:
                                seen[(src, tgt, "reaction")] += 1
                    else:
                        for k in range(32):
                            src = 32 * q + (lane + k) % 32
                            seen[(tgt, src, "target")] += 1
                            seen[(src, tgt, "reaction")] += 1
    return exclusive, seen


def mixed_item(T, diag, planted=None):
    """The same for one item of the mixed kernel: (phase exclusivity, fold
    lanes right, Counter of (target, source, side))."""
    W, NC = T // 4, T // 2

    def chunk(p, t):
        return (t if planted == "phase" else 2 * p + t) % NC

    seen = Counter()
    exclusive, folds_ok = True, True
    for t in range(NC):
        exclusive &= len({chunk(p, t) for p in range(W)}) == W
        for p in range(W):
            cc = chunk(p, t)
            if diag and 2 * cc + 1 < 4 * p:
                continue  # wholly below the warp's entries
            for lane in range(32):
                for k in range(32):
                    m = (lane + k) % 32
                    if planted == "step":
                        m = (lane + 2 * k) % 32
                    if k == 16:  # the kernel folds lane l's sums into pair block (l + 16) mod 32
                        folds_ok &= m == (lane + 16) % 32
                    for a in range(4):
                        et = 128 * p + 32 * a + lane
                        for h in range(2):
                            es = 64 * cc + 2 * m + h
                            if diag and not et < es:
                                continue
                            seen[(et, es, "target")] += 1
                            seen[(es, et, "reaction")] += 1
    return exclusive, folds_ok, seen


def _check_off_diagonal(seen, B):
    want = {(i, j, side) for i in range(B) for j in range(B) for side in ("target", "reaction")}
    assert set(seen) == want
    assert set(seen.values()) == {1}


def _check_diagonal(seen, B):
    # every unordered pair {i, j}, i != j: body i gets j's pull once and j
    # gets i's once, whichever side of the pair evaluation carries it
    pull = Counter()
    for (x, y, _side), n in seen.items():
        assert x != y, "an entry met itself"
        pull[(x, y)] += n
    want = {(i, j) for i in range(B) for j in range(B) if i != j}
    assert set(pull) == want
    assert set(pull.values()) == {1}


@pytest.mark.parametrize("T", [8, 16])
def test_wide_fp64_schedule(T):
    ex, seen = wide_fp64_item(T, diag=False)
    assert ex
    _check_off_diagonal(seen, 32 * T)
    ex, seen = wide_fp64_item(T, diag=True)
    assert ex
    _check_diagonal(seen, 32 * T)


@pytest.mark.parametrize("T", [4, 8, 16])
def test_mixed_schedule(T):
    ex, folds, seen = mixed_item(T, diag=False)
    assert ex and folds
    _check_off_diagonal(seen, 32 * T)
    ex, folds, seen = mixed_item(T, diag=True)
    assert ex and folds
    _check_diagonal(seen, 32 * T)


def test_planted_schedule_errors_fail():
    # a phase rule under which the warps take the same chunk at the same time
    # (every pair is still met once: only the exclusivity check sees the race)
    ex, _, seen = mixed_item(8, diag=False, planted="phase")
    assert not ex
    _check_off_diagonal(seen, 256)
    # a step rule that meets some pair blocks twice and others never
    _, folds, seen = mixed_item(8, diag=False, planted="step")
    assert not folds
    with pytest.raises(AssertionError):
        _check_off_diagonal(seen, 256)
    # a diagonal rule that also counts the pair in the other direction
    _, seen = wide_fp64_item(8, diag=False)
    with pytest.raises(AssertionError):
        _check_diagonal(seen, 256)


def item_rows(ns, B):
    """The partial rows each body of one system receives from the items of
    the pair-once kernels: the block pairs (I, J), I <= J, of blocks of B
    bodies; block I's sums go to row J of its bodies, block J's to row I, a
    diagonal item's (both sides) to row I."""
    nb = (ns + B - 1) // B
    got = Counter()
    for I in range(nb):
        for J in range(I, nb):
            for body in range(I * B, min(ns, (I + 1) * B)):
                got[(body, J)] += 1  # block I's sums (on a diagonal item, with block J's)
            if I != J:
                for body in range(J * B, min(ns, (J + 1) * B)):
                    got[(body, I)] += 1
    return nb, got


@pytest.mark.parametrize("ns,B", [(1283, 64), (1536, 64), (10425, 256), (4096, 4096), (5003, 128), (129, 128)])
def test_every_body_has_one_value_per_row(ns, B):
    nb, got = item_rows(ns, B)
    assert set(got) == {(body, row) for body in range(ns) for row in range(nb)}
    assert set(got.values()) == {1}
