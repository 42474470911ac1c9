"""Generalized real Schur form of a matrix pair (the QZ algorithm): the
generalized case the paper treats in its remarks (Sec. 1: (A, B) ->
Hessenberg-triangular (H, R) -> generalized Schur form (S, T); Sec. 2.1: the
iteration and LAPACK's infinite-eigenvalue convention; Sec. 2.2: shifts from
the trailing 2x2 pair, the bulge v = (H R^-1 - l1)(H R^-1 - l2) e1, left
reflectors plus right reflectors that restore R's triangular form; Sec. 3.2
and Sec. 3.4: infinite eigenvalues chased to the upper-left corner of the
active block).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Notation: the pair (H, T) is reduced in place; Q and Z accumulate the left
and right transformations so that the input pair equals
(Q H Z^T, Q T Z^T) throughout.  Every rotation and reflector is applied
directly, one at a time, to full rows (columns from the transform's first
column to n-1) and full columns (rows 0 to the transform's last row), which
gives the full generalized Schur form.
"""

import numpy as np

from .householder import reflector
from .qr import U, smlnum


# ------------------------------------------------------------ elementary

def rot_rows(M, i, k, c, s, cols):
    """Rows (i, k) <- [c s; -s c] (rows i, k) on the given columns."""
    x = M[i, cols].copy()
    y = M[k, cols].copy()
    M[i, cols] = c * x + s * y
    M[k, cols] = -s * x + c * y


def rot_cols(M, i, k, c, s, rows):
    """Columns (i, k) <- (columns i, k) [c -s; s c] on the given rows, i.e.
    new column i = c x_i + s x_k, new column k = -s x_i + c x_k."""
    x = M[rows, i].copy()
    y = M[rows, k].copy()
    M[rows, i] = c * x + s * y
    M[rows, k] = -s * x + c * y


def rot_zeroing_second(a, b):
    """(c, s) with -s a + c b = 0: a left rotation of rows (i, k) that zeroes
    the entry b of row k (the pair (a, b) becomes (hypot(a, b), 0))."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def rot_zeroing_first(a, b):
    """(c, s) with c a + s b = 0: a right rotation of columns (i, k) that
    zeroes the entry a of column i in that row."""
    if a == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return b / r, -a / r


def apply_left(M, v, tau, rows, cols):
    if tau == 0.0:
        return
    blk = M[rows, cols]
    M[rows, cols] = blk - tau * np.outer(v, v @ blk)


def apply_right(M, v, tau, rows, cols):
    if tau == 0.0:
        return
    blk = M[rows, cols]
    M[rows, cols] = blk - tau * np.outer(blk @ v, v)


def right_reflector_for_row(r):
    """(w, tau) with r (I - tau w w^T) = (0, .., 0, *): the reflector of the
    reversed row, reversed (w[-1] = 1)."""
    v, tau, _ = reflector(np.asarray(r, dtype=np.float64)[::-1])
    return v[::-1].copy(), tau


# ------------------------------------------------ Hessenberg-triangular

def hessenberg_triangular(A, B):
    """(H, R, Q, Z) with A = Q H Z^T, B = Q R Z^T, H upper Hessenberg and R
    upper triangular (Sec. 1 remark; Golub & Van Loan Alg. 7.7.1): a
    Householder QR of B applied to A, then Givens rotations that zero A's
    entries below the subdiagonal column by column from the bottom, each
    followed by the right rotation that removes the fill it makes in R."""
    H = np.array(A, dtype=np.float64, copy=True)
    R = np.array(B, dtype=np.float64, copy=True)
    n = H.shape[0]
    Q = np.eye(n)
    Z = np.eye(n)
    for j in range(n - 1):
        v, tau, beta = reflector(R[j:, j])
        apply_left(R, v, tau, slice(j, n), slice(j, n))
        apply_left(H, v, tau, slice(j, n), slice(0, n))
        apply_right(Q, v, tau, slice(0, n), slice(j, n))
        R[j, j] = beta
        R[j + 1:, j] = 0.0
    for j in range(n - 2):
        for i in range(n - 1, j + 1, -1):
            c, s = rot_zeroing_second(H[i - 1, j], H[i, j])
            rot_rows(H, i - 1, i, c, s, slice(j, n))
            rot_rows(R, i - 1, i, c, s, slice(i - 1, n))
            rot_cols(Q, i - 1, i, c, s, slice(0, n))
            H[i, j] = 0.0
            c, s = rot_zeroing_first(R[i, i - 1], R[i, i])
            rot_cols(R, i - 1, i, c, s, slice(0, i + 1))
            rot_cols(H, i - 1, i, c, s, slice(0, n))
            rot_cols(Z, i - 1, i, c, s, slice(0, n))
            R[i, i - 1] = 0.0
    return H, R, Q, Z


# ------------------------------------------------------------ the sweep

def shifted_first_column(H, T, lo, hi, ssum, sprod):
    """The first column of (M - l1)(M - l2) = M^2 - ssum M + sprod I,
    M = H T^-1, restricted to rows lo..lo+2 (Sec. 2.2 remark).  M is upper
    Hessenberg, so M e1 has two entries and M^2 e1 three."""
    m0 = np.zeros(3)
    m1 = np.zeros(3)
    # columns lo and lo+1 of M on rows lo..lo+2
    m0[:2] = H[lo:lo + 2, lo] / T[lo, lo]
    m1[:3] = (H[lo:lo + 3, lo + 1] - m0 * T[lo, lo + 1]) / T[lo + 1, lo + 1]
    msq = m0[0] * m0 + m0[1] * m1          # M (M e1)
    v = msq - ssum * m0
    v[0] += sprod
    return v


def trailing_shift_pair(H, T, lo, hi):
    """(ssum, sprod) = trace and determinant of the trailing 2x2 of
    M = H T^-1 on the block lo..hi (its eigenvalues are those of the trailing
    2x2 pair when the block is larger than 2x2: Sec. 2.2 remark)."""
    a = max(lo, hi - 2)
    Ti = np.linalg.inv(T[a:hi + 1, a:hi + 1])
    M = H[hi - 1:hi + 1, a:hi + 1] @ Ti[:, -2:]
    return M[0, 0] + M[1, 1], M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]


def exceptional_shift_pair(H, T, lo, hi):
    """Ad-hoc double shift after 10 iterations without deflation (the QR
    iteration's EISPACK constants applied to M = H T^-1's trailing entries;
    the paper is silent)."""
    mhh = H[hi, hi] / T[hi, hi]
    s = abs(H[hi, hi - 1] / T[hi - 1, hi - 1]) + (abs(H[hi - 1, hi - 2] / T[hi - 2, hi - 2]) if hi - 2 >= lo else 0.0)
    a = mhh + 0.75 * s
    return 2.0 * a, a * a + 0.4375 * s * s


def qz_sweep(H, T, Q, Z, lo, hi, ssum, sprod):
    """One double-shift QZ sweep on the unreduced block lo..hi (hi - lo >= 2)
    (Sec. 2.2 remark; Golub & Van Loan Alg. 7.7.2): for k = lo..hi-2 a left
    3x3 reflector moves the bulge of H one column down, then a right 3x3
    reflector zeroes T[k+2, k:k+2] and a right 2x2 reflector zeroes
    T[k+1, k]; the last position uses 2x2 reflectors."""
    n = H.shape[0]
    x = shifted_first_column(H, T, lo, hi, ssum, sprod)
    for k in range(lo, hi - 1):
        # left: rows k..k+2
        v, tau, beta = reflector(x)
        c0 = max(k - 1, lo) if k > lo else lo
        apply_left(H, v, tau, slice(k, k + 3), slice(c0, n))
        apply_left(T, v, tau, slice(k, k + 3), slice(k, n))
        apply_right(Q, v, tau, slice(0, n), slice(k, k + 3))
        if k > lo:
            H[k, k - 1] = beta
            H[k + 1, k - 1] = 0.0
            H[k + 2, k - 1] = 0.0
        # right: zero T[k+2, k], T[k+2, k+1]
        w, tw = right_reflector_for_row(T[k + 2, k:k + 3])
        rmax = min(k + 3, hi)
        apply_right(H, w, tw, slice(0, rmax + 1), slice(k, k + 3))
        apply_right(T, w, tw, slice(0, k + 3), slice(k, k + 3))
        apply_right(Z, w, tw, slice(0, n), slice(k, k + 3))
        T[k + 2, k] = 0.0
        T[k + 2, k + 1] = 0.0
        # right: zero T[k+1, k]
        w, tw = right_reflector_for_row(T[k + 1, k:k + 2])
        apply_right(H, w, tw, slice(0, rmax + 1), slice(k, k + 2))
        apply_right(T, w, tw, slice(0, k + 2), slice(k, k + 2))
        apply_right(Z, w, tw, slice(0, n), slice(k, k + 2))
        T[k + 1, k] = 0.0
        x = H[k + 1:k + 4, k].copy() if k + 3 <= hi else H[k + 1:k + 3, k].copy()
    # last position: rows hi-1, hi
    k = hi - 1
    v, tau, beta = reflector(x[:2])
    apply_left(H, v, tau, slice(k, k + 2), slice(k - 1, n))
    apply_left(T, v, tau, slice(k, k + 2), slice(k, n))
    apply_right(Q, v, tau, slice(0, n), slice(k, k + 2))
    H[k, k - 1] = beta
    H[k + 1, k - 1] = 0.0
    w, tw = right_reflector_for_row(T[k + 1, k:k + 2])
    apply_right(H, w, tw, slice(0, hi + 1), slice(k, k + 2))
    apply_right(T, w, tw, slice(0, k + 2), slice(k, k + 2))
    apply_right(Z, w, tw, slice(0, n), slice(k, k + 2))
    T[k + 1, k] = 0.0


# --------------------------------------------------- infinite eigenvalues

def chase_infinite_to_top(H, T, Q, Z, lo, hi, j):
    """T[j, j] = 0 on the block lo..hi: move the zero up the diagonal of T to
    (lo, lo) and deflate it there (Sec. 3.2 / 3.4: infinite eigenvalues are
    chased to the upper-left corner of the active block).  For i = j..lo+1
    a right rotation of columns (i-1, i) zeroes T[i-1, i-1] (the zero moves
    up; T stays triangular because row i of T is zero in both columns), then a
    left rotation of rows (i, i+1) removes the fill H[i+1, i-1].  At the top a
    left rotation of rows (lo, lo+1) zeroes H[lo+1, lo]: the 1x1 pair
    (H[lo, lo], 0) splits off."""
    n = H.shape[0]
    for i in range(j, lo, -1):
        c, s = rot_zeroing_first(T[i - 1, i - 1], T[i - 1, i])
        rot_cols(T, i - 1, i, c, s, slice(0, i + 1))
        rot_cols(H, i - 1, i, c, s, slice(0, min(i + 1, hi) + 1))
        rot_cols(Z, i - 1, i, c, s, slice(0, n))
        T[i - 1, i - 1] = 0.0
        T[i, i - 1] = 0.0
        if i + 1 <= hi:
            c, s = rot_zeroing_second(H[i, i - 1], H[i + 1, i - 1])
            rot_rows(H, i, i + 1, c, s, slice(i - 1, n))
            rot_rows(T, i, i + 1, c, s, slice(i, n))
            rot_cols(Q, i, i + 1, c, s, slice(0, n))
            H[i + 1, i - 1] = 0.0
            T[i + 1, i] = 0.0
    if lo < hi:
        c, s = rot_zeroing_second(H[lo, lo], H[lo + 1, lo])
        rot_rows(H, lo, lo + 1, c, s, slice(lo, n))
        rot_rows(T, lo, lo + 1, c, s, slice(lo, n))
        rot_cols(Q, lo, lo + 1, c, s, slice(0, n))
        H[lo + 1, lo] = 0.0
        T[lo, lo] = 0.0
        T[lo + 1, lo] = 0.0


# ---------------------------------------------------------- 2x2 blocks

def pair_eigs_2x2(S2, T2):
    """Eigenvalues of the 2x2 pair (S2, T2), T2 upper triangular and
    nonsingular: the roots of det(S2 - l T2) = 0, i.e. the eigenvalues of
    S2 T2^-1 (a 2x2 matrix, closed form)."""
    M = S2 @ np.linalg.inv(T2)
    tr = M[0, 0] + M[1, 1]
    det = M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]
    disc = 0.25 * tr * tr - det
    if disc >= 0.0:
        r = np.sqrt(disc)
        return np.array([0.5 * tr + r, 0.5 * tr - r]), False
    r = np.sqrt(-disc)
    return np.array([0.5 * tr + 1j * r, 0.5 * tr - 1j * r]), True


def standardize_pair_block(H, T, Q, Z, k):
    """The 2x2 diagonal block pair at rows/columns k, k+1, with T's block
    nonsingular.  Real eigenvalues: split it (a right rotation whose first
    column is an eigenvector of the pair, then the left rotation that makes
    T triangular again; S's subdiagonal entry then vanishes).  Complex
    eigenvalues: make T's block diagonal with positive entries (its 2x2
    singular value decomposition applied from both sides), LAPACK's
    standardised form.  Returns True for a complex pair."""
    n = H.shape[0]
    S2 = H[k:k + 2, k:k + 2].copy()
    T2 = T[k:k + 2, k:k + 2].copy()
    lam, cpx = pair_eigs_2x2(S2, T2)
    if not cpx:
        l1 = lam[0]
        K = S2 - l1 * T2
        # null vector of K: orthogonal to its larger row
        row = K[0] if np.hypot(*K[0]) >= np.hypot(*K[1]) else K[1]
        x = np.array([-row[1], row[0]])
        if np.hypot(*x) == 0.0:
            x = np.array([1.0, 0.0])
        x = x / np.hypot(*x)
        c, s = x[0], x[1]          # first column of the rotation = x
        rot_cols(H, k, k + 1, c, s, slice(0, k + 2))
        rot_cols(T, k, k + 1, c, s, slice(0, k + 2))
        rot_cols(Z, k, k + 1, c, s, slice(0, n))
        c, s = rot_zeroing_second(T[k, k], T[k + 1, k])
        rot_rows(H, k, k + 1, c, s, slice(k, n))
        rot_rows(T, k, k + 1, c, s, slice(k, n))
        rot_cols(Q, k, k + 1, c, s, slice(0, n))
        H[k + 1, k] = 0.0
        T[k + 1, k] = 0.0
        return False
    Uo, sv, Vt = np.linalg.svd(T2)
    Vo = Vt.T
    # left Uo^T on rows k, k+1; right Vo on columns k, k+1
    H[k:k + 2, k:n] = Uo.T @ H[k:k + 2, k:n]
    T[k:k + 2, k:n] = Uo.T @ T[k:k + 2, k:n]
    Q[:, k:k + 2] = Q[:, k:k + 2] @ Uo
    H[0:k + 2, k:k + 2] = H[0:k + 2, k:k + 2] @ Vo
    T[0:k + 2, k:k + 2] = T[0:k + 2, k:k + 2] @ Vo
    Z[:, k:k + 2] = Z[:, k:k + 2] @ Vo
    T[k, k], T[k, k + 1], T[k + 1, k], T[k + 1, k + 1] = sv[0], 0.0, 0.0, sv[1]
    return True


# -------------------------------------------------------------- driver

def ht_subdiag_negligible(H, k, n):
    """|H[k, k-1]| <= max(u (|H[k-1, k-1]| + |H[k, k]|), smlnum): the
    standard small-subdiagonal test (the QR iteration's, Sec. 2.1)."""
    return abs(H[k, k - 1]) <= max(U * (abs(H[k - 1, k - 1]) + abs(H[k, k])), smlnum(n))


def qz(H0, T0, Q0=None, Z0=None, maxit_factor=30):
    """(S, T, Q, Z, alphar, alphai, beta, info) for the Hessenberg-triangular
    pair (H0, T0): (S, T) = Q^T (H0, T0) Z in generalized real Schur form
    (Q, Z accumulated into Q0, Z0 when given).  Eigenvalue i is
    (alphar_i + i alphai_i) / beta_i; beta_i = 0 for an infinite eigenvalue.
    T's diagonal entries with |T_ii| <= u ||T0||_F are set to zero (LAPACK's
    convention, Sec. 2.1 remark).  info = 0, or 1 + the top row of a block
    that did not converge within maxit_factor * (its size) iterations."""
    S = np.triu(np.array(H0, dtype=np.float64, copy=True), -1)
    T = np.triu(np.array(T0, dtype=np.float64, copy=True))
    n = S.shape[0]
    Q = np.eye(n) if Q0 is None else np.array(Q0, dtype=np.float64, copy=True)
    Z = np.eye(n) if Z0 is None else np.array(Z0, dtype=np.float64, copy=True)
    tthr = U * np.linalg.norm(T)
    hi = n - 1
    its = 0
    info = 0
    while hi >= 0:
        # deflation: the top of the unreduced block ending at hi
        lo = hi
        while lo > 0 and not ht_subdiag_negligible(S, lo, n):
            lo -= 1
        if lo > 0:
            S[lo, lo - 1] = 0.0
        # infinite eigenvalues in the block
        inf_j = -1
        for j in range(lo, hi + 1):
            if abs(T[j, j]) <= tthr:
                T[j, j] = 0.0
                if inf_j < 0:
                    inf_j = j
        if inf_j >= 0 and hi > lo:
            chase_infinite_to_top(S, T, Q, Z, lo, hi, inf_j)
            its = 0
            continue
        size = hi - lo + 1
        if size == 1:
            hi -= 1
            its = 0
            continue
        if size == 2:
            standardize_pair_block(S, T, Q, Z, lo)
            hi -= 2
            its = 0
            continue
        its += 1
        if its > maxit_factor * size:
            info = lo + 1
            break
        if its % 10 == 0:
            ssum, sprod = exceptional_shift_pair(S, T, lo, hi)
        else:
            ssum, sprod = trailing_shift_pair(S, T, lo, hi)
        qz_sweep(S, T, Q, Z, lo, hi, ssum, sprod)
    alphar, alphai, beta = eig_from_gschur(S, T)
    return S, T, Q, Z, alphar, alphai, beta, info


def eig_from_gschur(S, T):
    """(alphar, alphai, beta) of a standardised generalized Schur pair: a 1x1
    block gives (S_kk, 0, T_kk) with the sign making beta >= 0; a complex 2x2
    block (T diagonal, positive) gives alpha_k = lambda T_kk and
    alpha_{k+1} = conj(lambda) T_{k+1,k+1}, lambda with positive imaginary
    part first (LAPACK's convention)."""
    n = S.shape[0]
    ar, ai, be = np.zeros(n), np.zeros(n), np.zeros(n)
    k = 0
    while k < n:
        if k + 1 < n and S[k + 1, k] != 0.0:
            lam, _ = pair_eigs_2x2(S[k:k + 2, k:k + 2], T[k:k + 2, k:k + 2])
            l1 = lam[0] if np.imag(lam[0]) > 0 else lam[1]
            ar[k], ai[k], be[k] = np.real(l1) * T[k, k], np.imag(l1) * T[k, k], T[k, k]
            ar[k + 1], ai[k + 1], be[k + 1] = np.real(l1) * T[k + 1, k + 1], -np.imag(l1) * T[k + 1, k + 1], \
                T[k + 1, k + 1]
            k += 2
        else:
            sgn = -1.0 if T[k, k] < 0.0 else 1.0
            ar[k], ai[k], be[k] = sgn * S[k, k], 0.0, sgn * T[k, k]
            k += 1
    return ar, ai, be


def eigenvalues(alphar, alphai, beta):
    """Complex eigenvalues (inf for beta = 0)."""
    out = np.empty(len(beta), dtype=complex)
    for i in range(len(beta)):
        out[i] = complex(alphar[i], alphai[i]) / beta[i] if beta[i] != 0.0 else complex(np.inf, 0.0)
    return out


def gschur_structure_errors(S, T):
    """Violations of the standardised generalized Schur form: S quasi upper
    triangular with 2x2 blocks only for complex pairs, T upper triangular,
    T's 2x2 diagonal blocks diagonal with positive entries."""
    n = S.shape[0]
    errs = []
    if np.any(np.tril(S, -2) != 0.0):
        errs.append("S below subdiagonal")
    if np.any(np.tril(T, -1) != 0.0):
        errs.append("T below diagonal")
    for k in range(n - 1):
        if S[k + 1, k] != 0.0:
            if k + 2 < n and S[k + 2, k + 1] != 0.0:
                errs.append(f"adjacent subdiagonals at {k}")
            if T[k, k + 1] != 0.0 or T[k, k] <= 0.0 or T[k + 1, k + 1] <= 0.0:
                errs.append(f"T block at {k} not positive diagonal")
            lam, cpx = pair_eigs_2x2(S[k:k + 2, k:k + 2], T[k:k + 2, k:k + 2])
            if not cpx:
                errs.append(f"real pair in 2x2 block at {k}")
    return errs
