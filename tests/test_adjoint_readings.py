"""The two facts the eigenvalue adjoint's large-order path is built on,
checked on the CPU with the oracle's Schur forms and eigenvectors (no GPU):

1. With R the reversal permutation, S' = R S^T R is again a standardised
   quasi-triangular matrix with the same 2x2 blocks (mirrored), and its right
   eigenvectors, reversed, are the vectors w of S^T (S^T w = lambda w) that
   the oracle computes by forward substitution: the large-order path gets
   the left vectors from the right-vector solver this way.
2. With X the right vectors (upper quasi-triangular in LAPACK's real format)
   and P the scaled w's (lower, one extra entry per pair), G = P X^T is zero
   above its second superdiagonal, and the column-block / row-chunk bounds
   the path's GEMMs use (k >= j0 - 1, k <= i1 for G; k >= j0 - 2 for Z G)
   drop only zero terms.
"""

import numpy as np
import pytest

from oracle import metrics, qr
from paper_2007_03576_gb300 import inputs


def _schur(n, seed):
    H = inputs.hessrand(n, [seed, 31])
    S, Z, wr, wi, info = qr.schur(H)
    assert info == 0
    return S, Z, wr, wi


def _real_format(X, wi):
    """Complex right vectors (one per eigenvalue) -> LAPACK's real format."""
    n = X.shape[0]
    Xr = np.zeros((n, n))
    k = 0
    while k < n:
        Xr[:, k] = X[:, k].real
        if wi[k] > 0 and k + 1 < n:
            Xr[:, k + 1] = X[:, k].imag
            k += 2
        else:
            k += 1
    return Xr


@pytest.mark.parametrize("n,seed", [(9, 1), (40, 2), (75, 3)])
def test_reversed_transpose_gives_the_left_vectors(n, seed):
    S, _, wr, wi = _schur(n, seed)
    assert np.sum(wi > 0) >= 1
    Sp = S[::-1, ::-1].T.copy()
    assert metrics.schur_structure_errors(Sp) == []
    wrp, wip = qr.eig_from_schur(Sp)
    assert np.array_equal(wrp, wr[::-1])
    assert np.array_equal(wip, np.where(wi[::-1] == 0, 0.0, -wi[::-1]))
    lam, X, W = metrics.eigvecs_quasi_triangular(S)
    lamp, Xp, Wp = metrics.eigvecs_quasi_triangular(Sp)
    for k in range(n):
        if wi[k] < 0:
            continue
        # eigenvalue k of S sits at n-1-k of S' (a pair (k, k+1) at (n-2-k, n-1-k))
        kp = n - 1 - k if wi[k] == 0 else n - 2 - k
        assert abs(lamp[kp] - lam[k]) <= 1e-12 * max(1.0, abs(lam[k]))
        w_rev = Xp[::-1, kp]
        # same vector up to a complex scale
        c = np.vdot(W[:, k], w_rev)
        assert abs(abs(c) - np.linalg.norm(W[:, k]) * np.linalg.norm(w_rev)) <= 1e-10 * abs(c)
        assert np.linalg.norm(S.T @ w_rev - lam[k] * w_rev) <= 1e-12 * np.linalg.norm(S) * np.linalg.norm(w_rev)


@pytest.mark.parametrize("n,seed", [(30, 4), (70, 5)])
def test_g_zero_pattern_and_product_bounds(n, seed):
    S, Z, wr, wi = _schur(n, seed)
    lam, X, W = metrics.eigvecs_quasi_triangular(S)
    Xr = _real_format(X, wi)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    c = np.sum(W * X, axis=0)
    P = np.zeros((n, n))
    k = 0
    while k < n:
        if wi[k] > 0 and k + 1 < n:
            e = (np.conj(g[k]) + g[k + 1]) / c[k]
            P[:, k] = (e * W[:, k]).real
            P[:, k + 1] = -(e * W[:, k]).imag
            k += 2
        else:
            P[:, k] = (np.conj(g[k]) / c[k] * W[:, k]).real
            k += 1
    # P lower with one extra entry per pair, X upper with one per pair
    assert np.all(np.triu(P, 2) == 0.0) and np.all(np.tril(Xr, -2) == 0.0)
    G = P @ Xr.T
    # the same G as the direct sum over eigenvalues of Re(conj(g_k)/c_k w_k x_k^T)
    Gd = np.real((W * (np.conj(g) / c)[None, :]) @ X.T)
    assert np.max(np.abs(G - Gd)) <= 1e-11 * np.max(np.abs(Gd))
    assert np.max(np.abs(np.triu(G, 3))) <= 1e-13 * np.max(np.abs(G))
    # blocked products with small blocks: columns of 4, rows in chunks of 8
    Gb = np.zeros((n, n))
    for j0 in range(0, n, 4):
        j1, k0 = min(n, j0 + 4), max(0, j0 - 1)
        for i0 in range(max(0, j0 - 2), n, 8):
            i1 = min(n, i0 + 8)
            k1 = min(n, i1 + 1)
            Gb[i0:i1, j0:j1] = P[i0:i1, k0:k1] @ Xr[j0:j1, k0:k1].T
    assert np.max(np.abs(Gb - G)) <= 1e-13 * np.max(np.abs(G))
    T = np.zeros((n, n))
    for j0 in range(0, n, 4):
        j1, k0 = min(n, j0 + 4), max(0, j0 - 2)
        T[:, j0:j1] = Z[:, k0:] @ Gb[k0:, j0:j1]
    assert np.max(np.abs(T - Z @ G)) <= 1e-13 * np.max(np.abs(Z @ G))
