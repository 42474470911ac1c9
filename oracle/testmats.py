"""Matrices with known spectra for pinning the oracle.  Test infrastructure only.

* ``companion``  -- upper Hessenberg companion matrix of a polynomial with
                    prescribed roots (its eigenvalues are those roots).
* ``cyclic``     -- the n-cycle permutation matrix (eigenvalues: the n-th
                    roots of unity); already upper Hessenberg, and a matrix on
                    which Francis / AED shifts stall without exceptional
                    shifts.
* ``prescribed`` -- Q blockdiag(...) Q^T, Hessenberg-reduced, with real
                    eigenvalues in [-10, 10] and 2x2 blocks [[a, b], [-b, a]]
                    (optionally plus a strictly upper-triangular U[-1,1] part).
* ``syn``        -- the paper's syn_n family (Sec. 5.3 item 2).
"""

import numpy as np

from .householder import hessenberg_reduce


def companion(roots):
    """Companion matrix of prod (z - r_i) in upper Hessenberg form: first row
    -c_1 .. -c_n of the monic coefficients, ones on the subdiagonal.  The
    coefficients come from numpy.poly (a library primitive)."""
    c = np.real_if_close(np.poly(np.asarray(roots)))
    c = np.real(c)
    n = len(c) - 1
    H = np.zeros((n, n))
    H[0, :] = -c[1:]
    H[np.arange(1, n), np.arange(0, n - 1)] = 1.0
    return H


def cyclic(n):
    """n-cycle permutation matrix (H[i+1, i] = 1, H[0, n-1] = 1)."""
    H = np.zeros((n, n))
    H[np.arange(1, n), np.arange(0, n - 1)] = 1.0
    H[0, n - 1] = 1.0
    return H


def haar_orthogonal(n, rng):
    """Haar-distributed orthogonal matrix: Q factor of a Gaussian matrix with
    the signs fixed by diag(R) > 0 (numpy QR as a library primitive)."""
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))[None, :]


def prescribed_blocks(n, rng, nonnormal=False):
    """(T, eigenvalues) of the prescribed-spectrum family before the
    similarity: T = D (+ N), D block diagonal with n/2 real eigenvalues
    ~ U[-10, 10] and n/4 blocks [[a, b], [-b, a]], a ~ U[-10, 10],
    b ~ U[0.5, 10]; N strictly upper U[-1, 1] (non-normal variant), zero
    inside the 2x2 blocks.  Draws the same numbers as ``prescribed``."""
    T, lam, _ = _prescribed_parts(n, rng, nonnormal)
    return T, lam


def prescribed(n, rng, nonnormal=False, reduce=None):
    """(H, eigenvalues): n/2 real eigenvalues ~ U[-10, 10] and n/4 complex
    pairs a +- i b, a ~ U[-10, 10], b ~ U[0.5, 10] as 2x2 blocks
    [[a, b], [-b, a]]; optional strictly upper U[-1, 1] part (non-normal);
    A = Q D Q^T with Haar Q, then reduced to Hessenberg form by Householder
    reflectors (``reduce``: A -> H, default the oracle's unblocked
    reduction; any orthogonal reduction keeps the spectrum)."""
    T, lam, rng = _prescribed_parts(n, rng, nonnormal)
    Q = haar_orthogonal(n, rng)
    A = Q @ T @ Q.T
    if reduce is None:
        H, _ = hessenberg_reduce(A)
    else:
        H = reduce(A)
    return H, np.array(lam)


def _prescribed_parts(n, rng, nonnormal):
    npairs = n // 4
    nreal = n - 2 * npairs
    D = np.zeros((n, n))
    lam = []
    re = rng.uniform(-10, 10, nreal)
    for i in range(nreal):
        D[i, i] = re[i]
        lam.append(re[i])
    a = rng.uniform(-10, 10, npairs)
    b = rng.uniform(0.5, 10, npairs)
    for k in range(npairs):
        j = nreal + 2 * k
        D[j, j] = D[j + 1, j + 1] = a[k]
        D[j, j + 1] = b[k]
        D[j + 1, j] = -b[k]
        lam += [a[k] + 1j * b[k], a[k] - 1j * b[k]]
    if nonnormal:
        N = np.triu(rng.uniform(-1, 1, (n, n)), 1)
        for k in range(npairs):  # keep the 2x2 blocks intact
            j = nreal + 2 * k
            N[j, j + 1] = 0.0
        D = D + N
    return D, np.array(lam), rng


def syn(n, rng):
    """syn_n (Sec. 5.3 item 2): known eigenvalues +-1, +-3, +-5, ...; random
    disjoint adjacent pairs (lam_i, lam_{i+1}) are lifted to
    Re(lam_i) +- i |Re(lam_i)| until half of the eigenvalues are complex;
    they sit on the diagonal (2x2 blocks [[r, |r|], [-|r|, r]]) of a random
    upper-triangular U[-1, 1] matrix; A = Qbar S Qbar^T with one random
    Householder reflector Qbar; returns (H, eigenvalues) with H the
    Householder Hessenberg form of A."""
    base = np.empty(n)
    base[0::2] = 2 * np.arange((n + 1) // 2) + 1
    base[1::2] = -(2 * np.arange(n // 2) + 1)
    S = np.triu(rng.uniform(-1, 1, (n, n)), 1)
    lam = base.astype(complex)
    used = np.zeros(n, dtype=bool)
    ncomplex = 0
    order = rng.permutation(n - 1)
    for i in order:
        if ncomplex >= n // 2:
            break
        if used[i] or used[i + 1]:
            continue
        used[i] = used[i + 1] = True
        r = base[i]
        lam[i] = r + 1j * abs(r)
        lam[i + 1] = r - 1j * abs(r)
        ncomplex += 2
    i = 0
    while i < n:
        if used[i]:
            r = lam[i].real
            S[i, i] = S[i + 1, i + 1] = r
            S[i, i + 1] = abs(r)
            S[i + 1, i] = -abs(r)
            i += 2
        else:
            S[i, i] = lam[i].real
            i += 1
    u = rng.standard_normal(n)
    Qb = np.eye(n) - 2.0 * np.outer(u, u) / (u @ u)
    H, _ = hessenberg_reduce(Qb @ S @ Qb.T)
    return H, lam
