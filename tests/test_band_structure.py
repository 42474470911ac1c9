"""Host-side checks of the chase schedule that the driver issues and of the
band of the chase windows' accumulated transforms.

The schedule comes from the library itself (schur_chase_schedule, the
function Solver::sweep launches from; no GPU needed): chains of bulges,
chain c started S launches after chain c - 1, each launch moving every chain
delta steps (Sec. 2.3/2.4, Fig. 3).  The checks:
  - every bulge passes every row of the active block exactly once, inside
    its window;
  - k_apply_u skips (16 x row-block) tiles of U that are structurally zero:
    the driver declares, for a window of a chain of nb bulges moved delta
    steps, the band  r - c <= 2 + 2 min(nb - 1, delta - 1)  and
    c - r <= delta + 1, checked by propagating the nonzero pattern of U
    through the window's reflectors (a reflector on rows/columns k..k+2
    couples them), including the first (bulge introduction) and last
    (bulges leaving) windows;
  - a chase step's right products miss the next step's windows (the
    three-stream overlap relies on it)."""

import ctypes

import numpy as np
import pytest

from paper_2007_03576_gb300 import _lib


def library_schedule(lo, hi, npairs, nbc):
    """[(launch, ws, we, tau0, tau1, pair0, nb)], kwin, delta of a sweep, from
    the library."""
    lib = _lib.load()
    count, kwin, delta = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.schur_chase_schedule(lo, hi, npairs, nbc, 0, None, ctypes.byref(count), None, None) == 0
    buf = (ctypes.c_int * (7 * max(1, count.value)))()
    assert lib.schur_chase_schedule(lo, hi, npairs, nbc, count.value, buf, ctypes.byref(count),
                                    ctypes.byref(kwin), ctypes.byref(delta)) == 0
    recs = [tuple(buf[7 * i:7 * i + 7]) for i in range(count.value)]
    return recs, kwin.value, delta.value


def schedule(lo, hi, npairs, nbc_req):
    recs, kwin, delta = library_schedule(lo, hi, npairs, nbc_req)
    for s, ws, we, tau0, tau1, pair0, nb in recs:
        yield ws, we, tau0, tau1, nb, delta


@pytest.mark.parametrize("n,npairs,nbc,lo", [(300, 8, 4, 0), (400, 30, 10, 7), (260, 4, 1, 0), (500, 64, 32, 0),
                                              (700, 48, 24, 3), (20000, 64, 16, 0), (5000, 1024, 0, 0)])
def test_schedule_moves_every_bulge_through_every_row_once(n, npairs, nbc, lo):
    """Sec. 2.3: each bulge is introduced at the top of the active block and
    chased off its bottom: bulge j of a chain sits at row lo + tau - 3 j at
    chain-local step tau, and every row k in [lo, hi - 1] is visited once,
    inside the window of the launch that moves it; chains share no launch
    window rows; every pair is used."""
    hi = n - 1
    recs, kwin, delta = library_schedule(lo, hi, npairs, nbc)
    seen = {}
    by_launch = {}
    for s, ws, we, tau0, tau1, pair0, nb in recs:
        assert we - ws + 1 <= kwin and 1 <= tau1 - tau0 <= delta
        by_launch.setdefault(s, []).append((ws, we))
        for tau in range(tau0, tau1):
            for j in range(nb):
                k = lo + tau - 3 * j
                if lo <= k <= hi - 1:
                    key = (pair0 + j, k)
                    assert key not in seen, key
                    seen[key] = s
                    assert ws <= k and k + min(3, hi - k + 1) - 1 <= we
                    if k > lo:
                        assert ws <= k - 1
    assert len(seen) == npairs * (hi - lo)
    for wins in by_launch.values():
        wins.sort()
        for (a0, b0), (a1, b1) in zip(wins, wins[1:]):
            assert b0 < a1


def pattern(lo, hi, ws, we, tau0, tau1, nb):
    L = we - ws + 1
    P = np.eye(L, dtype=bool)
    for tau in range(tau0, tau1):
        for j in range(nb):            # bottom bulge first, as in the chase
            k = lo + tau - 3 * j
            if lo <= k <= hi - 1:
                nr = min(3, hi - k + 1)
                kl = k - ws
                rows = P[:, kl:kl + nr].any(axis=1)
                P[np.ix_(rows, np.arange(kl, kl + nr))] = True
    return P


@pytest.mark.parametrize("n,npairs,nbc", [(300, 8, 4), (400, 30, 10), (260, 4, 1), (500, 64, 32), (700, 48, 24)])
def test_chase_transform_band(n, npairs, nbc):
    for ws, we, tau0, tau1, nb, delta in schedule(0, n - 1, npairs, nbc):
        P = pattern(0, n - 1, ws, we, tau0, tau1, nb)
        r, c = np.nonzero(P)
        assert np.max(r - c) <= 2 + 2 * min(nb - 1, delta - 1)
        assert np.max(c - r) <= delta + 1


def range_rule(lo, hi, ws, we, tau0, tau1, nb):
    """The chase kernel's bookkeeping of U's nonzero rows: column c's rows lie
    in [ulo[c], uhi[c]], initially [c, c]; a reflector on columns kl..kl+nr-1
    gives all of them the union of their ranges.  Yields, before each step's
    right products, the ranges next to the structural pattern of U."""
    L = we - ws + 1
    ulo, uhi = np.arange(L), np.arange(L)
    P = np.eye(L, dtype=bool)
    for tau in range(tau0, tau1):
        for j in range(nb):
            k = lo + tau - 3 * j
            if lo <= k <= hi - 1:
                nr = min(3, hi - k + 1)
                kl = k - ws
                cols = np.arange(kl, kl + nr)
                a, b = ulo[cols].min(), uhi[cols].max()
                ulo[cols], uhi[cols] = a, b
                rows = P[:, cols].any(axis=1)
                P[np.ix_(rows, cols)] = True
        yield ulo.copy(), uhi.copy(), P.copy()


@pytest.mark.parametrize("n,npairs,nbc", [(300, 8, 4), (400, 30, 10), (260, 4, 1), (500, 64, 32), (700, 32, 16)])
def test_chase_u_row_ranges_cover_nonzeros(n, npairs, nbc):
    """The right products of the chase touch only rows ulo..uhi of U's
    columns: after every step those ranges contain every structural nonzero,
    and they are narrower than the window (the saving the kernel takes)."""
    saved = total = 0
    for ws, we, tau0, tau1, nb, delta in schedule(0, n - 1, npairs, nbc):
        L = we - ws + 1
        for ulo, uhi, P in range_rule(0, n - 1, ws, we, tau0, tau1, nb):
            r, c = np.nonzero(P)
            assert np.all(r >= ulo[c]) and np.all(r <= uhi[c])
            saved += int(np.sum(L - (uhi - ulo + 1)))
            total += L * L
    assert saved > 0.2 * total


def test_chase_u_row_ranges_numeric():
    """The same with numbers: U accumulated from random 3x3 reflectors of one
    window schedule has no nonzero outside the tracked ranges."""
    rng = np.random.default_rng(5)
    for ws, we, tau0, tau1, nb, delta in schedule(0, 299, 16, 8):
        L = we - ws + 1
        U = np.eye(L)
        ulo, uhi = np.arange(L), np.arange(L)
        for tau in range(tau0, tau1):
            for j in range(nb):
                k = tau - 3 * j
                if 0 <= k <= 298:
                    nr = min(3, 299 - k + 1)
                    kl = k - ws
                    cols = np.arange(kl, kl + nr)
                    a, b = ulo[cols].min(), uhi[cols].max()
                    ulo[cols], uhi[cols] = a, b
                    v = rng.standard_normal(nr)
                    Pm = np.eye(nr) - 2.0 * np.outer(v, v) / (v @ v)
                    U[:, cols] = U[:, cols] @ Pm
        r, c = np.nonzero(U)
        assert np.all(r >= ulo[c]) and np.all(r <= uhi[c])


def launches(lo, hi, npairs, nbc_req):
    """The windows of each chase launch of a sweep: [[(ws, we), ...], ...]
    in launch order, from the library's schedule."""
    recs, _, _ = library_schedule(lo, hi, npairs, nbc_req)
    out = {}
    for s, ws, we, *_ in recs:
        out.setdefault(s, []).append((ws, we))
    return [out[s] for s in sorted(out)]


@pytest.mark.parametrize("n,npairs,nbc,lo", [(20000, 64, 16, 0), (5000, 32, 16, 37), (3000, 32, 8, 0),
                                              (2000, 64, 4, 11), (700, 10, 3, 0), (20000, 128, 32, 5)])
def test_right_products_miss_the_next_chase_step(n, npairs, nbc, lo):
    """A chase step's right products (rows 0..ws-1 of columns ws..we of each
    window) touch nothing the next chase step reads (its windows), so they run
    beside it on another stream.  The next step's left products (rows of its
    windows, columns to the right) do meet them where a following chain's rows
    cross the columns of the chain ahead: that is why they wait."""
    hi = n - 6
    sch = launches(lo, hi, npairs, nbc)
    meets_left = 0
    for s in range(len(sch) - 1):
        for ws, we in sch[s]:
            for ws2, we2 in sch[s + 1]:
                # right products of (ws, we) vs window (ws2, we2) of the next launch
                rows_meet = ws2 < ws
                cols_meet = not (we2 < ws or ws2 > we)
                assert not (rows_meet and cols_meet)
                # left products of (ws2, we2): rows ws2..we2, columns > we2
                if ws2 < ws and we2 < we:
                    meets_left += 1
    if npairs > nbc:
        assert meets_left > 0
