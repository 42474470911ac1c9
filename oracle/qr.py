"""Multishift QR with aggressive early deflation -- the plain CPU FP64 oracle.

Test infrastructure only (see ``oracle/__init__``).  Written from the paper
(Myllykoski, ACM TOMS 2021): Sec. 2.1 (outline of the iteration), Sec. 2.2
(double-implicit-shift step, Fig. 1), Sec. 2.3 (tightly-coupled multishift
sweep, Fig. 2), Sec. 2.5 (aggressive early deflation, Fig. 4) and Sec. 5.6
(deflation conditions).  Everything is applied in "full Schur form" mode:
every similarity transformation acts on whole rows/columns of H and on all
rows of the accumulated Z, so that on exit H_in = Z S Z^T.

Conventions
-----------
* Matrices are numpy float64 arrays, 0-based indices; an active (unreduced)
  block is the inclusive index range [lo, hi].
* ``U`` is the paper's unit roundoff u = 2^-52 (Sec. 5.4) and ``NU`` is the
  paper's nu = smallest number whose reciprocal does not overflow
  (Sec. 5.6), read as DBL_MIN = 2^-1022.
* A shift pair is stored as (sum, product) = (s1 + s2, s1 * s2); for a
  complex conjugate pair both are real.

Where the paper is silent the reading taken is stated at the function that
applies it.
"""

import math
from dataclasses import dataclass

import numpy as np

from .householder import reflector, apply_left, apply_right

U = 2.0 ** -52
NU = 2.0 ** -1022
MAX_DEPTH = 2   # windows of windows are reduced by Francis double-shift QR


def smlnum(n):
    """nu * (n / u): the absolute floor of the LAPACK-style tests (Sec. 5.6)."""
    return NU * (n / U)


@dataclass
class Params:
    """Tuning knobs.  ns / nw = 0 selects the default table ``default_ns_nw``.

    deflation: "lapack" (Sec. 5.6 item 1, used in all of the paper's
    experiments), "norm" (item 2, norm-stable) or "fixed" (item 3, threshold
    ``thold``).
    """
    ns: int = 0
    nw: int = 0
    nmin: int = 75
    nibble: int = 14
    deflation: str = "lapack"
    thold: float = 0.0
    exc_period: int = 6
    nwin_francis: int = 0    # AED windows up to max(nmin, this) use Francis QR (0: nmin, LAPACK's rule)
    swap_tol: float = 10.0   # a swap is rejected when its residual exceeds swap_tol * u * ||A||_F
    recompute_shifts: bool = False  # shifts from the trailing ns x ns block when AED leaves <= ns/2
    normH: float = 0.0  # ||H||_F of the input, set by ``schur``
    depth: int = 0      # AED recursion depth (0 = the input matrix)

    def for_window(self):
        """Parameters for the recursive QR inside an AED window: same
        deflation mode, default shift/window table, one level deeper."""
        return Params(ns=0, nw=0, nmin=self.nmin, nibble=self.nibble, deflation=self.deflation,
                      thold=self.thold, exc_period=self.exc_period, nwin_francis=self.nwin_francis,
                      swap_tol=self.swap_tol, recompute_shifts=self.recompute_shifts,
                      normH=self.normH, depth=self.depth + 1)


def default_ns_nw(m):
    """Default (number of shifts, AED window) for an active block of size m.

    The paper gives no table (it sizes windows by tiles, Sec. 3.2); this
    reading follows the growth of LAPACK's defaults and the configurations of
    the workloads (n = 256: 8 shifts, window 32; n = 20000: 128-256 shifts,
    window ~3% of n).
    """
    if m < 150:
        return 8, 24
    if m < 590:
        return 8, 32
    if m < 3000:
        return 64, 96
    if m < 6000:
        return 64, 128
    ns = 256
    return ns, min(1024, max(3 * ns // 2, int(round(0.03 * m))))


# --------------------------------------------------------------------------
# 2x2 blocks: eigenvalues and standardisation (eq. 2by2_blocks)
# --------------------------------------------------------------------------

def eig2x2(a, b, c, d):
    """Eigenvalues of [[a, b], [c, d]] as ((re1, im1), (re2, im2)); for a
    complex pair im1 > 0 > im2."""
    p = 0.5 * (a - d)
    disc = p * p + b * c
    mid = 0.5 * (a + d)
    if disc >= 0.0:
        r = math.sqrt(disc)
        return (mid + r, 0.0), (mid - r, 0.0)
    r = math.sqrt(-disc)
    return (mid, r), (mid, -r)


def standardize_2x2(a, b, c, d):
    """Rotation G = [[cs, -sn], [sn, cs]] putting [[a, b], [c, d]] in the
    standard form of a real Schur factor (eq. ``2by2_blocks``): a complex
    pair gives equal diagonal entries and off-diagonal entries of opposite
    sign; real eigenvalues give an upper-triangular block.

    Reading (the paper prints only the condition on the eigenvalues): the
    rotation is taken from the 2x2 Schur factorisation itself.  Real case:
    the first column of G is a unit eigenvector of the eigenvalue
    (a+d)/2 + sign(a-d) r.  Complex case: G^T A G has diagonal difference
    (a-d) cos 2t + (b+c) sin 2t, which the angle t = atan2(-(a-d), b+c)/2
    makes zero.  Returns (cs, sn, [[a', b'], [c', d']]).
    """
    if c == 0.0:
        return 1.0, 0.0, np.array([[a, b], [0.0, d]])
    p = 0.5 * (a - d)
    disc = p * p + b * c
    if disc >= 0.0:
        r = math.sqrt(disc)
        z = p + math.copysign(r, p)          # lambda1 - d
        lam1 = d + z
        u1 = (z, c)
        u2 = (b, lam1 - a)
        u = u1 if abs(u1[0]) + abs(u1[1]) >= abs(u2[0]) + abs(u2[1]) else u2
        nrm = math.hypot(u[0], u[1])
        cs, sn = u[0] / nrm, u[1] / nrm
    else:
        t = 0.5 * math.atan2(-(a - d), b + c)
        cs, sn = math.cos(t), math.sin(t)
    G = np.array([[cs, -sn], [sn, cs]])
    B = G.T @ np.array([[a, b], [c, d]]) @ G
    if disc >= 0.0:
        B[1, 0] = 0.0
        return cs, sn, B
    m = 0.5 * (B[0, 0] + B[1, 1])
    B[0, 0] = B[1, 1] = m
    if B[0, 1] * B[1, 0] < 0.0:
        return cs, sn, B
    # Rounding turned the pair real (b'c' >= 0 with equal diagonal):
    # triangularise the rotated block and compose the two rotations.
    cs2, sn2, B2 = standardize_2x2(B[0, 0], B[0, 1], B[1, 0], B[1, 1])
    return cs * cs2 - sn * sn2, sn * cs2 + cs * sn2, B2


def standardize_block(H, Z, k):
    """Standardise the decoupled 2x2 diagonal block H[k:k+2, k:k+2] and apply
    its rotation to the rest of the rows (columns k..n-1), the rest of the
    columns (rows 0..k+1) and to Z."""
    n = H.shape[0]
    cs, sn, B = standardize_2x2(H[k, k], H[k, k + 1], H[k + 1, k], H[k + 1, k + 1])
    if cs == 1.0 and sn == 0.0:
        return
    G = np.array([[cs, -sn], [sn, cs]])
    if k + 2 < n:
        H[k:k + 2, k + 2:] = G.T @ H[k:k + 2, k + 2:]
    if k > 0:
        H[:k, k:k + 2] = H[:k, k:k + 2] @ G
    Z[:, k:k + 2] = Z[:, k:k + 2] @ G
    H[k:k + 2, k:k + 2] = B


# --------------------------------------------------------------------------
# Deflation conditions (Sec. 5.6)
# --------------------------------------------------------------------------

def subdiag_negligible(H, k, lo, hi, P, n):
    """Vigilant-deflation test for the subdiagonal entry H[k, k-1] (Sec. 2.1
    "vigilant deflation"; Sec. 5.6 lists one test per deflation mode).

    LAPACK-style mode: the paper states that the vigilant checks mirror
    LAPACK 3.9.0.  Reading: the entry is negligible if it is below
    nu*n/u, or below u*(|h_{k-1,k-1}| + |h_kk|) *and* passes the
    Ahues-Tisseur refinement |h21| |h12| <= u |h22| |h11 - h22| (both sides
    scaled by max(|h22|, |h11-h22|) + max(|h21|, |h12|)).
    """
    h21 = abs(H[k, k - 1])
    if P.deflation == "norm":
        return h21 <= U * P.normH
    if P.deflation == "fixed":
        return h21 <= P.thold
    sml = smlnum(n)
    if h21 <= sml:
        return True
    tst = abs(H[k - 1, k - 1]) + abs(H[k, k])
    if tst == 0.0:
        if k - 2 >= lo:
            tst += abs(H[k - 1, k - 2])
        if k + 1 <= hi:
            tst += abs(H[k + 1, k])
    if h21 > U * tst:
        return False
    h12 = abs(H[k - 1, k])
    d = abs(H[k - 1, k - 1] - H[k, k])
    h22 = abs(H[k, k])
    ab, ba = max(h21, h12), min(h21, h12)
    aa, bb = max(h22, d), min(h22, d)
    s = aa + ab
    return ba * (ab / s) <= max(sml, U * (bb * (aa / s)))


def spike_deflatable(T, spike, j, bs, P, n):
    """AED deflation test (Sec. 5.6) of the diagonal block of T ending at row
    j (size bs = 1 or 2) against the spike entries spike[j-bs+1 .. j]."""
    if bs == 1:
        s = abs(spike[j])
        if P.deflation == "norm":
            return s <= U * P.normH
        if P.deflation == "fixed":
            return s <= P.thold
        return s <= max(smlnum(n), U * abs(T[j, j]))
    s = max(abs(spike[j]), abs(spike[j - 1]))
    if P.deflation == "norm":
        return s <= U * P.normH
    if P.deflation == "fixed":
        return s <= P.thold
    hhat = math.sqrt(abs(T[j, j] * T[j - 1, j - 1])) + math.sqrt(abs(T[j - 1, j] * T[j, j - 1]))
    return s <= max(smlnum(n), U * hhat)


# --------------------------------------------------------------------------
# Bulge chasing (Sec. 2.2 and 2.3)
# --------------------------------------------------------------------------

def shift_vector(H, lo, hi, ssum, sprod):
    """First column of (H - s1 I)(H - s2 I) restricted to rows lo..lo+2 of the
    active block (Sec. 2.2: v = (H - l1 I)(H - l2 I) e_1)."""
    h00, h01 = H[lo, lo], H[lo, lo + 1]
    h10, h11 = H[lo + 1, lo], H[lo + 1, lo + 1]
    x = h00 * h00 + h01 * h10 - ssum * h00 + sprod
    y = h10 * (h00 + h11 - ssum)
    if lo + 2 <= hi:
        return np.array([x, y, h10 * H[lo + 2, lo + 1]])
    return np.array([x, y])


def bulge_step(H, Z, lo, hi, k, pair):
    """Move one bulge by one position: build the reflector at row k (from the
    shift vector when k == lo, else from column k-1, rows k..k+2) and apply
    it to the whole of rows k..k+2 (columns k..n-1), to rows 0..min(k+3, hi)
    of columns k..k+2, and to Z.  At k = hi-1 the reflector has order 2 (the
    bulge leaves the block)."""
    n = H.shape[0]
    nr = min(3, hi - k + 1)
    if k == lo:
        x = shift_vector(H, lo, hi, pair[0], pair[1])[:nr]
    else:
        x = H[k:k + nr, k - 1].copy()
    v, tau, beta = reflector(x)
    if k > lo:
        H[k, k - 1] = beta
        H[k + 1:k + nr, k - 1] = 0.0
    rows = slice(k, k + nr)
    apply_left(H, v, tau, rows, slice(k, n))
    apply_right(H, v, tau, slice(0, min(k + 3, hi) + 1), rows)
    apply_right(Z, v, tau, slice(0, Z.shape[0]), rows)


def double_shift_sweep(H, Z, lo, hi, ssum, sprod):
    """One Francis double-implicit-shift sweep on the unreduced block [lo, hi]
    (Sec. 2.2, Fig. 1): introduce the bulge with the shift pair and chase it
    off the bottom with overlapping 3x3 reflectors."""
    for k in range(lo, hi):
        bulge_step(H, Z, lo, hi, k, (ssum, sprod))


def multishift_sweep(H, Z, lo, hi, pairs):
    """Tightly-coupled multishift sweep (Sec. 2.3, Fig. 2), reflectors applied
    directly (no window accumulation).

    Bulge j (0-based, in the order of ``pairs``) is introduced at the top once
    bulge j-1 has moved three rows down, i.e. at global step t = 3j; at step t
    it sits at row k = lo + t - 3j.  Within a step the bulges are moved
    bottom (j = 0) to top, the order in which introducing the bulges one at a
    time and chasing each just far enough leaves every reflector's input
    unchanged.  The windowed GPU chase applies the same reflectors, grouped
    into windows and accumulated.
    """
    nb = len(pairs)
    steps = (hi - lo) + 3 * (nb - 1)
    for t in range(steps):
        for j in range(nb):
            k = lo + t - 3 * j
            if lo <= k <= hi - 1:
                bulge_step(H, Z, lo, hi, k, pairs[j])


def exceptional_pairs(H, ktop, kbot, npairs):
    """Ad-hoc shifts used when the iteration stalls (reading: the paper is
    silent; EISPACK's exceptional shift of Wilkinson & Reinsch): for
    i = kbot, kbot-2, ...: with s = |h_{i,i-1}| + |h_{i-1,i-2}| and
    a = h_ii + 0.75 s, the complex pair a +- i sqrt(0.4375) s, i.e.
    (sum, product) = (2a, a^2 + 0.4375 s^2)."""
    pairs = []
    i = kbot
    while len(pairs) < npairs and i > ktop:
        s = abs(H[i, i - 1]) + (abs(H[i - 1, i - 2]) if i - 2 >= ktop else 0.0)
        a = H[i, i] + 0.75 * s
        pairs.append((2.0 * a, a * a + 0.4375 * s * s))
        i -= 2
    return pairs


# --------------------------------------------------------------------------
# Small QR (Francis double shift) -- the "small Schur" task of Sec. 3.2
# --------------------------------------------------------------------------

def find_ktop(H, lo, hi, P, n):
    """Scan the subdiagonal of [lo, hi] upward from hi; the first negligible
    entry is set to zero and its row returned (else lo)."""
    for k in range(hi, lo, -1):
        if H[k, k - 1] == 0.0 or subdiag_negligible(H, k, lo, hi, P, n):
            H[k, k - 1] = 0.0
            return k
    return lo


def francis_qr(H, Z, lo, hi, P, n=None):
    """Reduce the block [lo, hi] to real Schur form with Francis double-shift
    sweeps (Sec. 2.2): Francis shifts from the trailing 2x2, an exceptional
    pair every 10th iteration on the same block, vigilant deflation by
    ``subdiag_negligible``; deflated 2x2 blocks are standardised.

    Returns 0, or i+1 if the iteration limit 30*max(10, m) was hit while
    rows lo..i were still unreduced.
    """
    if n is None:
        n = H.shape[0]
    i = hi
    itmax = 30 * max(10, hi - lo + 1)
    total = 0
    while i >= lo:
        its = 0
        while True:
            l = find_ktop(H, lo, i, P, n)
            if l >= i - 1:
                break
            its += 1
            total += 1
            if total > itmax:
                return i + 1
            if its % 10 == 0:
                (ssum, sprod), = exceptional_pairs(H, l, i, 1)
            else:
                a, b, c, d = H[i - 1, i - 1], H[i - 1, i], H[i, i - 1], H[i, i]
                ssum, sprod = a + d, a * d - b * c
            double_shift_sweep(H, Z, l, i, ssum, sprod)
        if l == i:
            i -= 1
        else:
            standardize_block(H, Z, i - 1)
            i -= 2
    return 0


# --------------------------------------------------------------------------
# Eigenvalue reordering (Sec. 2.5 step 2)
# --------------------------------------------------------------------------

def _solve_complete_pivot(K, rhs, sml):
    """Gaussian elimination with complete pivoting for the small Kronecker
    system of the Sylvester equation; a pivot below ``sml`` is replaced by
    ``sml`` (the perturbation used by Bai & Demmel when the two blocks share
    an eigenvalue)."""
    K = K.copy()
    b = rhs.copy()
    m = K.shape[0]
    perm = list(range(m))
    for i in range(m):
        sub = np.abs(K[i:, i:])
        r, c = np.unravel_index(np.argmax(sub), sub.shape)
        r += i
        c += i
        K[[i, r]] = K[[r, i]]
        b[[i, r]] = b[[r, i]]
        K[:, [i, c]] = K[:, [c, i]]
        perm[i], perm[c] = perm[c], perm[i]
        if abs(K[i, i]) < sml:
            K[i, i] = sml
        for rr in range(i + 1, m):
            f = K[rr, i] / K[i, i]
            K[rr, i:] -= f * K[i, i:]
            b[rr] -= f * b[i]
    y = np.zeros(m)
    for i in range(m - 1, -1, -1):
        y[i] = (b[i] - K[i, i + 1:] @ y[i + 1:]) / K[i, i]
    x = np.zeros(m)
    for i in range(m):
        x[perm[i]] = y[i]
    return x


def block_size_at(T, j):
    """Size (1 or 2) of the diagonal block of the quasi-triangular T that
    starts at row j."""
    return 2 if j + 1 < T.shape[0] and T[j + 1, j] != 0.0 else 1


def swap_adjacent(T, V, j, p, q, tol=10.0):
    """Swap the adjacent diagonal blocks T[j:j+p, j:j+p] (p x p) and
    T[j+p:j+p+q, j+p:j+p+q] (q x q) of the quasi-triangular T by an orthogonal
    similarity, accumulating into V (direct swapping of Bai & Demmel 1993,
    cited by the paper in Sec. 2.5).

    With A = [[A11, A12], [0, A22]], the solution X of the Sylvester equation
    A11 X - X A22 = A12 makes the columns of [-X; I] span the invariant
    subspace of A22; the orthogonal factor Q of their QR factorisation swaps
    the blocks.  The swap is rejected (T and V untouched, returns False) when
    the new (2,1) block of Q^T A Q exceeds max(tol u ||A||_F, nu n / u),
    tol = 10 (reading of the paper's "too ill-conditioned", Sec. 3.5.3;
    Bai & Demmel's weak stability test).  Swapped 2x2 blocks are
    re-standardised.
    """
    nT = T.shape[0]
    m = p + q
    A = T[j:j + m, j:j + m].copy()
    A11, A12, A22 = A[:p, :p], A[:p, p:], A[p:, p:]
    K = np.kron(np.eye(q), A11) - np.kron(A22.T, np.eye(p))
    sml = max(U * np.max(np.abs(K)), smlnum(nT))
    x = _solve_complete_pivot(K, A12.reshape(-1, order="F"), sml)
    X = x.reshape(p, q, order="F")
    W = np.vstack([-X, np.eye(q)])
    Q = np.eye(m)
    for c in range(q):
        v, tau, beta = reflector(W[c:, c])
        apply_left(W, v, tau, slice(c, m), slice(c, q))
        apply_right(Q, v, tau, slice(0, m), slice(c, m))
    A2 = Q.T @ A @ Q
    if np.linalg.norm(A2[q:, :q]) > max(tol * U * np.linalg.norm(A), smlnum(nT)):
        return False
    blk = slice(j, j + m)
    T[blk, j:] = Q.T @ T[blk, j:]
    T[:j + m, blk] = T[:j + m, blk] @ Q
    V[:, blk] = V[:, blk] @ Q
    T[j + q:j + m, j:j + q] = 0.0
    if q == 2:
        standardize_block(T, V, j)
    if p == 2:
        standardize_block(T, V, j + q)
    return True


def move_block_up(T, V, ifst, ilst, p=None, tol=10.0):
    """Move the diagonal block starting at row ifst up so that it starts at
    row ilst (ilst <= ifst, a block boundary) by adjacent swaps.  The block is
    moved as a unit of its original size p even if it splits on the way.
    Returns False (T stays in Schur form) if a swap is rejected."""
    if p is None:
        p = block_size_at(T, ifst)
    here = ifst
    while here > ilst:
        q = 2 if here >= 2 and here - 2 >= ilst and T[here - 1, here - 2] != 0.0 else 1
        if not swap_adjacent(T, V, here - q, q, p, tol):
            return False
        here -= q
    return True


# --------------------------------------------------------------------------
# Aggressive early deflation (Sec. 2.5, Fig. 4)
# --------------------------------------------------------------------------

def block_eigs(T, lo, hi):
    """Eigenvalues of the 1x1 / 2x2 diagonal blocks of T[lo:hi, lo:hi], top to
    bottom, as a list of (re, im); a 2x2 block contributes its pair with
    the positive imaginary part first."""
    out = []
    j = lo
    while j < hi:
        if j + 1 < hi and T[j + 1, j] != 0.0:
            e1, e2 = eig2x2(T[j, j], T[j, j + 1], T[j + 1, j], T[j + 1, j + 1])
            out += [e1, e2]
            j += 2
        else:
            out.append((T[j, j], 0.0))
            j += 1
    return out


def aed(H, Z, ktop, kbot, nw, P, n=None):
    """One AED step on the trailing nw x nw window of the active block
    [ktop, kbot] (Sec. 2.5):

    1. the window T is copied out and reduced to Schur form T = V T_S V^T by
       recursive QR: this driver when nw exceeds the crossover
       max(nmin, nwin_francis), Francis double-shift QR otherwise, and always
       Francis for the window of a window.  Reading: the paper says
       "recursive application of the QR algorithm" (Sec. 2.5) and implements
       the small AED task with LAPACK's sequential QR (Sec. 3.2, the small
       AED task calls DHSEQR), whose AED uses the double-shift routine for
       windows of at most NMIN rows and the recursive multishift routine
       above (NMIN = 75 by default, a machine-dependent tunable), with the
       windows of the recursive level reduced by the double-shift routine.
       The default nwin_francis = 0 takes that rule with NMIN = nmin; a
       larger nwin_francis moves the crossover as a tuning of NMIN does;
    2. with s = h_{kwtop, kwtop-1} the spike is s * V[0, :]; candidates are
       tested bottom-up (``spike_deflatable``); a failed block is moved to
       the top of the unevaluated part (``move_block_up``); a rejected swap
       halts the reordering (greedy rule, Sec. 3.5.4);
    3. if at least one eigenvalue deflated, the spike of the undeflated part
       is reflected onto its first entry and the undeflated part is returned
       to Hessenberg form by Householder reflectors; the window is copied
       back and V is applied to the rest of H and to Z.  With no deflation
       nothing is written back (Sec. 2.5, last paragraph).

    Returns (nd, candidates): the number of deflated eigenvalues and the
    eigenvalues of the undeflated blocks (top to bottom) -- the shifts of the
    next sweep.
    """
    if n is None:
        n = H.shape[0]
    kwtop = kbot - nw + 1
    s = 0.0 if kwtop == ktop else H[kwtop, kwtop - 1]
    T = np.triu(H[kwtop:kbot + 1, kwtop:kbot + 1], -1).copy()
    V = np.eye(nw)
    Pw = P.for_window()
    if nw <= max(P.nmin, P.nwin_francis) or Pw.depth >= MAX_DEPTH:
        info = francis_qr(T, V, 0, nw - 1, Pw, nw)
    else:
        info = qr_block(T, V, 0, nw - 1, Pw, nw)
    ns = nw
    ilst = info  # an unconverged top part is treated as undeflatable
    while ilst < ns:
        bs = 2 if ns >= 2 and T[ns - 1, ns - 2] != 0.0 else 1
        spike = s * V[0, :]
        if spike_deflatable(T, spike, ns - 1, bs, P, n):
            ns -= bs
            continue
        if not move_block_up(T, V, ns - bs, ilst, bs, P.swap_tol):
            break
        ilst += bs
    nd = nw - ns
    candidates = block_eigs(T, info, ns)
    if nd == 0:
        return 0, candidates
    spike = s * V[0, :ns].copy()
    top = 0.0
    if ns == 1:
        top = spike[0]
    elif ns > 1 and s != 0.0:
        v, tau, beta = reflector(spike)
        apply_left(T, v, tau, slice(0, ns), slice(0, nw))
        apply_right(T, v, tau, slice(0, nw), slice(0, ns))
        apply_right(V, v, tau, slice(0, nw), slice(0, ns))
        top = beta
        for j in range(ns - 2):
            v, tau, beta = reflector(T[j + 1:ns, j])
            apply_left(T, v, tau, slice(j + 1, ns), slice(j, nw))
            apply_right(T, v, tau, slice(0, nw), slice(j + 1, ns))
            apply_right(V, v, tau, slice(0, nw), slice(j + 1, ns))
            T[j + 1, j] = beta
            T[j + 2:ns, j] = 0.0
    if kwtop > ktop:
        H[kwtop, kwtop - 1] = top
        H[kwtop + 1:kbot + 1, kwtop - 1] = 0.0
    H[kwtop:kbot + 1, kwtop:kbot + 1] = np.triu(T, -1)
    if kbot + 1 < H.shape[1]:
        H[kwtop:kbot + 1, kbot + 1:] = V.T @ H[kwtop:kbot + 1, kbot + 1:]
    if kwtop > 0:
        H[:kwtop, kwtop:kbot + 1] = H[:kwtop, kwtop:kbot + 1] @ V
    Z[:, kwtop:kbot + 1] = Z[:, kwtop:kbot + 1] @ V
    return nd, candidates


def recomputed_candidates(H, ktop, kbot, ns, P, n):
    """Shift recomputation after AED (reading of Sec. 5, the comment on the
    residuals: LAPACK recomputes the shifts after an AED step under certain
    conditions, and the same is planned as an option in the paper's
    library).  The condition and the recomputation follow LAPACK's
    multishift driver: when AED has left at most ns/2 undeflated
    candidates, the candidates are replaced by the eigenvalues of the
    trailing r x r principal submatrix of the active block [ktop, kbot]
    (r = min(ns, 160, rows of the block); 160 rows is what one thread block
    of the GPU path holds), computed by double-shift QR on a copy (top to
    bottom).  Returns None when that QR hits its iteration limit (the AED
    candidates are kept)."""
    m = min(ns, 160, kbot - ktop + 1)
    ks = kbot - m + 1
    T = np.triu(H[ks:kbot + 1, ks:kbot + 1], -1).copy()
    if francis_qr(T, np.eye(m), 0, m - 1, P.for_window(), m):
        return None
    return block_eigs(T, 0, m)


def pairs_from_candidates(cands, npairs):
    """Shift pairs for the next sweep from the AED candidates (reading: the
    paper says the failed candidates become the shifts, Sec. 2.5; take the
    bottom-most ones, keep complex conjugates together, pair real shifts in
    order of appearance and drop an unpaired real one).  Returned bottom-most
    first; pair 0 drives the first bulge introduced."""
    pairs = []
    pending = None
    i = len(cands) - 1
    while i >= 0 and len(pairs) < npairs:
        re, im = cands[i]
        if im != 0.0:
            # the pair occupies cands[i-1], cands[i]
            pairs.append((2.0 * re, re * re + im * im))
            i -= 2
            continue
        if pending is None:
            pending = re
        else:
            pairs.append((pending + re, pending * re))
            pending = None
        i -= 1
    return pairs


# --------------------------------------------------------------------------
# The driver (Sec. 2.1)
# --------------------------------------------------------------------------

@dataclass
class Stats:
    aed: int = 0
    sweeps: int = 0
    francis: int = 0
    deflated_by_aed: int = 0
    recomputed: int = 0


def qr_block(H, Z, ilo, ihi, P, n=None, stats=None):
    """Reduce the block [ilo, ihi] of H to real Schur form (Sec. 2.1): repeat
    { find the bottom unreduced block [ktop, kbot]; if it is 1x1 or 2x2,
    deflate it; if it has at most nmin rows, finish it with Francis
    double-shift QR; else run AED; unless AED deflated more than nibble % of
    its window (then AED is repeated), run a multishift sweep with the
    failed candidates as shifts (exceptional shifts every exc_period-th
    iteration without deflation) }.

    Returns 0, or kbot+1 of the block that hit the iteration limit
    30*max(10, m) (Sec. 2.1: "... or an iteration limit is reached").
    """
    if n is None:
        n = H.shape[0]
    kbot = ihi
    itmax = 30 * max(10, ihi - ilo + 1)
    it = 0
    ndfl = 1
    while kbot >= ilo:
        ktop = find_ktop(H, ilo, kbot, P, n)
        m = kbot - ktop + 1
        if m == 1:
            kbot -= 1
            ndfl = 1
            continue
        if m == 2:
            standardize_block(H, Z, ktop)
            kbot -= 2
            ndfl = 1
            continue
        if m <= P.nmin:
            info = francis_qr(H, Z, ktop, kbot, P, n)
            if stats is not None:
                stats.francis += 1
            if info:
                return info
            kbot = ktop - 1
            ndfl = 1
            continue
        it += 1
        if it > itmax:
            return kbot + 1
        ns_max, nw = default_ns_nw(m)
        if P.ns:
            ns_max = P.ns
        if P.nw:
            nw = P.nw
        nw = min(nw, m)
        nd, cands = aed(H, Z, ktop, kbot, nw, P, n)
        if stats is not None:
            stats.aed += 1
            stats.deflated_by_aed += nd
        kbot -= nd
        ndfl = 1 if nd > 0 else ndfl + 1
        m = kbot - ktop + 1
        if m <= P.nmin:
            continue
        if nd > 0 and 100 * nd > P.nibble * nw:
            continue
        ns = min(ns_max, m - 1)
        ns -= ns % 2
        if ndfl % P.exc_period == 0:
            pairs = exceptional_pairs(H, ktop, kbot, ns // 2)
        else:
            if P.recompute_shifts and len(cands) <= ns // 2:
                rc = recomputed_candidates(H, ktop, kbot, ns, P, n)
                if rc is not None:
                    cands = rc
                    if stats is not None:
                        stats.recomputed += 1
            pairs = pairs_from_candidates(cands, ns // 2)
            if not pairs:
                a, b, c, d = H[kbot - 1, kbot - 1], H[kbot - 1, kbot], H[kbot, kbot - 1], H[kbot, kbot]
                pairs = [(a + d, a * d - b * c)]
        multishift_sweep(H, Z, ktop, kbot, pairs)
        if stats is not None:
            stats.sweeps += 1
    return 0


def eig_from_schur(S):
    """(wr, wi) of a standardised quasi-triangular S; a complex pair is
    stored with the positive imaginary part first."""
    n = S.shape[0]
    wr = np.zeros(n)
    wi = np.zeros(n)
    j = 0
    while j < n:
        if j + 1 < n and S[j + 1, j] != 0.0:
            (r1, i1), (r2, i2) = eig2x2(S[j, j], S[j, j + 1], S[j + 1, j], S[j + 1, j + 1])
            wr[j], wi[j], wr[j + 1], wi[j + 1] = r1, i1, r2, i2
            j += 2
        else:
            wr[j] = S[j, j]
            j += 1
    return wr, wi


def schur(H0, Z0=None, params=None, stats=None):
    """H0 (upper Hessenberg) -> (S, Z, wr, wi, info) with H0 = Z S Z^T.

    If Z0 is given the transformations are accumulated into it (Z = Z0 Z_QR),
    else Z starts as the identity.  info = 0 on success.
    """
    P = params if params is not None else Params()
    H = np.triu(np.array(H0, dtype=np.float64, copy=True), -1)
    n = H.shape[0]
    Z = np.eye(n) if Z0 is None else np.array(Z0, dtype=np.float64, copy=True)
    if P.normH == 0.0:
        P = Params(**{**P.__dict__, "normH": float(np.linalg.norm(H))})
    info = 0
    if n > 0:
        info = qr_block(H, Z, 0, n - 1, P, n, stats)
    H = np.triu(H, -1)
    wr, wi = eig_from_schur(H)
    return H, Z, wr, wi, info
