"""Host-side checks of how the single-matrix path splits each chase step's
products over its streams, on the decomposition the library itself issues
(schur_sweep_split_tasks; no GPU needed):

  - coverage: for every window, near + far left products cover exactly its
    rows x the columns right of it, right + cross products exactly the rows
    above it x its columns, each entry once;
  - within a step, the only rectangles that meet are a cross block and the
    left products of the window whose rows it lies on (the cross block runs
    after them on the far stream);
  - the next chase step's windows meet none of the step's far, cross or
    right products (they run beside it), and what they need of the step's
    left products is inside its near products (which the main stream
    finishes first).
"""

import ctypes

import numpy as np
import pytest

from paper_2007_03576_gb300 import _lib

NEAR, FAR, CROSS, RIGHT, ZK = 0, 1, 2, 3, 4


def split_tasks(n, lo, hi, npairs, nbc):
    lib = _lib.load()
    count = ctypes.c_int()
    assert lib.schur_sweep_split_tasks(n, lo, hi, npairs, nbc, 0, None, ctypes.byref(count)) == 0
    buf = (ctypes.c_int * (8 * max(1, count.value)))()
    assert lib.schur_sweep_split_tasks(n, lo, hi, npairs, nbc, count.value, buf, ctypes.byref(count)) == 0
    return [tuple(buf[8 * i:8 * i + 8]) for i in range(count.value)]


def windows(lo, hi, npairs, nbc):
    lib = _lib.load()
    count, kwin, delta = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.schur_chase_schedule(lo, hi, npairs, nbc, 0, None, ctypes.byref(count), None, None) == 0
    buf = (ctypes.c_int * (7 * max(1, count.value)))()
    assert lib.schur_chase_schedule(lo, hi, npairs, nbc, count.value, buf, ctypes.byref(count),
                                    ctypes.byref(kwin), ctypes.byref(delta)) == 0
    out = {}
    for i in range(count.value):
        s, ws, we = buf[7 * i], buf[7 * i + 1], buf[7 * i + 2]
        out.setdefault(s, []).append((ws, we))
    return out


def rect(rec):
    """(rows [a, b), cols [c, d)) of a record."""
    s, kind, chain, side, r0, c0, L, nvec = rec
    if side == 0:
        return (r0, r0 + L), (c0, c0 + nvec)
    return (r0, r0 + nvec), (c0, c0 + L)


def meets(x, y):
    (a0, a1), (b0, b1) = x
    (c0, c1), (d0, d1) = y
    return a0 < c1 and c0 < a1 and b0 < d1 and d0 < b1


CASES = [(300, 0, 299, 8, 4), (400, 7, 399, 30, 10), (700, 0, 699, 48, 24), (2000, 11, 1999, 64, 4),
         (3000, 0, 2999, 32, 8), (5000, 37, 4994, 128, 16)]


@pytest.mark.parametrize("n,lo,hi,npairs,nbc", CASES)
def test_split_products_cover_each_entry_once(n, lo, hi, npairs, nbc):
    recs = split_tasks(n, lo, hi, npairs, nbc)
    wins = windows(lo, hi, npairs, nbc)
    by_step = {}
    for r in recs:
        by_step.setdefault(r[0], []).append(r)
    assert sorted(by_step) == sorted(wins)
    for s, rs in by_step.items():
        ws_list = sorted(wins[s])
        for chain, (ws, we) in enumerate(wins[s]):
            mine = [r for r in rs if r[2] == chain and r[1] != ZK]
            left = np.zeros((we - ws + 1, n), dtype=int)
            above = np.zeros((ws, we - ws + 1), dtype=int)
            for r in mine:
                (a, b), (c, d) = rect(r)
                if r[1] in (NEAR, FAR):
                    assert a == ws and b == we + 1 and c > we
                    left[:, c:d] += 1
                else:
                    assert c == ws and d == we + 1 and b <= ws
                    above[a:b, :] += 1
            assert np.all(left[:, we + 1:] == 1) and np.all(left[:, :we + 1] == 0)
            assert np.all(above == 1)
            # cross blocks are exactly the rows of the windows above
            cross_rows = sorted((rect(r)[0]) for r in mine if r[1] == CROSS)
            assert cross_rows == [(a, b + 1) for a, b in ws_list if b < ws]
            assert [r for r in rs if r[2] == chain and r[1] == ZK]


@pytest.mark.parametrize("n,lo,hi,npairs,nbc", CASES)
def test_split_products_race_free(n, lo, hi, npairs, nbc):
    recs = split_tasks(n, lo, hi, npairs, nbc)
    wins = windows(lo, hi, npairs, nbc)
    by_step = {}
    for r in recs:
        if r[1] != ZK:
            by_step.setdefault(r[0], []).append(r)
    steps = sorted(by_step)
    for s in steps:
        rs = by_step[s]
        # within a step: only a cross block meets left products (those of the window above)
        for i in range(len(rs)):
            for j in range(i + 1, len(rs)):
                if meets(rect(rs[i]), rect(rs[j])):
                    kinds = sorted((rs[i][1], rs[j][1]))
                    assert kinds in ([NEAR, CROSS], [FAR, CROSS]), (s, rs[i], rs[j])
        # the next chase step's windows
        if s + 1 not in wins:
            continue
        for ws2, we2 in wins[s + 1]:
            box = ((ws2, we2 + 1), (ws2, we2 + 1))
            for r in rs:
                if r[1] in (FAR, CROSS, RIGHT):
                    assert not meets(rect(r), box), (s, r, (ws2, we2))
            # what the window needs of this step's left products is in the near products
            for chain, (ws, we) in enumerate(wins[s]):
                need = ((max(ws, ws2), min(we, we2) + 1), (we + 1, we2 + 1))
                if need[0][0] >= need[0][1] or need[1][0] >= need[1][1]:
                    continue
                near = [rect(r) for r in rs if r[1] == NEAR and r[2] == chain]
                assert near and near[0][1][0] <= need[1][0] and need[1][1] <= near[0][1][1]
