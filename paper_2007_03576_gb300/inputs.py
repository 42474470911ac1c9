"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module draws random numbers only; it holds none of the method's
arithmetic.  All generators use numpy's PCG64 (``numpy.random.default_rng``).

* ``hessrand(n, seed)`` -- the paper's hess_n family (Sec. 5.3 item 3):
  h_ij ~ N(0, 1) on and above the diagonal, h_{i+1,i} = sqrt(chi^2(n-i))
  (1-based i) on the subdiagonal, zero below.
* ``gaussian(n, seed)`` -- a dense N(0, 1) matrix (reduced to Hessenberg
  form by the oracle for the n = 256 workload).
* ``batch_sizes(count, lo, hi, seed)`` -- sizes uniform in [lo, hi] for the
  batched and differentiation workloads.
* ``ht_pair(n, seed, singular=0)`` -- a Hessenberg-triangular pair: H from
  hessrand, T upper triangular with N(0, 1) above the diagonal and
  chi(n-i+1) on it (the R factor of a Gaussian matrix's QR); ``singular``
  diagonal entries of T set to zero (infinite eigenvalues).

Matrices are returned as numpy arrays in row-major (C) order with the
mathematical layout H[i, j]; ``colmajor_bytes`` gives the column-major
copy that the C ABI expects (H^T in C order).
"""

import numpy as np


def hessrand(n, seed, dtype=np.float64):
    """Upper Hessenberg matrix of the hess_n family (Braman, Byers & Mathias
    generator as stated in Sec. 5.3): N(0,1) on and above the diagonal,
    chi(n-i) subdiagonal (1-based row i of the entry h_{i+1,i})."""
    rng = np.random.default_rng(seed)
    H = np.triu(rng.standard_normal((n, n)))
    if n > 1:
        dof = n - np.arange(1, n)          # n-1, n-2, ..., 1
        H[np.arange(1, n), np.arange(0, n - 1)] = np.sqrt(rng.chisquare(dof))
    return H.astype(dtype, copy=False)


def hessrand_colmajor(n, seed):
    """hessrand(n, seed) stored column-major: returns C-ordered H^T, whose
    memory is H in column-major order with leading dimension n.  Generated
    column by column so that n = 20000 needs no second n x n buffer."""
    rng = np.random.default_rng(seed)
    Ht = np.zeros((n, n))
    # same stream as hessrand: the upper triangle in row-major draw order
    # would require the full matrix; instead draw the full normal matrix in
    # row blocks and scatter the transpose.
    blk = 512
    for r0 in range(0, n, blk):
        r1 = min(n, r0 + blk)
        rows = rng.standard_normal((r1 - r0, n))
        for i in range(r0, r1):
            Ht[i:, i] = rows[i - r0, i:]
    if n > 1:
        dof = n - np.arange(1, n)
        sub = np.sqrt(rng.chisquare(dof))
        Ht[np.arange(0, n - 1), np.arange(1, n)] = sub
    return Ht


def gaussian(n, seed):
    """Dense n x n matrix with N(0, 1) entries."""
    return np.random.default_rng(seed).standard_normal((n, n))


def batch_sizes(count, lo, hi, seed):
    """count integers uniform in [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=count)


def batch_hessrand(sizes, seed):
    """List of hessrand matrices, matrix b drawn with seed (seed, b)."""
    return [hessrand(int(n), [seed, b]) for b, n in enumerate(sizes)]


def ht_pair(n, seed, singular=0):
    """(H, T) Hessenberg-triangular; T_ii = sqrt(chi^2(n - i)) (0-based i),
    N(0, 1) above; the first ``singular`` entries of a seeded choice of
    diagonal positions are set to zero."""
    rng = np.random.default_rng(list(np.atleast_1d(seed)) + [7])
    H = hessrand(n, seed)
    T = np.triu(rng.standard_normal((n, n)))
    T[np.arange(n), np.arange(n)] = np.sqrt(rng.chisquare(n - np.arange(n)))
    if singular:
        pos = rng.choice(n, size=singular, replace=False)
        T[pos, pos] = 0.0
    return H, T


def colmajor_bytes(A):
    """Column-major copy of A as a C-contiguous array (A^T in C order)."""
    return np.ascontiguousarray(np.asarray(A).T)
