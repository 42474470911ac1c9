"""Householder reflectors and the Householder Hessenberg reduction (oracle).

Test infrastructure only (see ``oracle/__init__``).

A reflector is P = I - tau * v v^T with v[0] = 1; P is symmetric and
orthogonal.  ``reflector(x)`` returns (v, tau, beta) with P x = beta e_1
(Golub & Van Loan, Matrix Computations, Sec. 5.1.2).  The 3x3 reflectors of
the bulge chase (paper Sec. 2.2: "a 3-by-3 Householder reflector ... such that
Q^T v is a multiple of e_1") are this routine applied to 3-vectors.
"""

import numpy as np


def reflector(x):
    """Return (v, tau, beta) with (I - tau v v^T) x = beta e_1 and v[0] = 1.

    beta = -sign(x_0) ||x||; if x[1:] is exactly zero the reflector is the
    identity (tau = 0, beta = x_0).
    """
    x = np.asarray(x, dtype=np.float64)
    v = np.zeros_like(x)
    v[0] = 1.0
    alpha = x[0]
    sigma = np.linalg.norm(x[1:]) if x.size > 1 else 0.0
    if sigma == 0.0:
        return v, 0.0, alpha
    beta = -np.copysign(np.hypot(alpha, sigma), alpha)
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, tau, beta


def apply_left(A, v, tau, rows, cols):
    """A[rows, cols] <- (I - tau v v^T) A[rows, cols]."""
    if tau == 0.0:
        return
    blk = A[rows, cols]
    A[rows, cols] = blk - tau * np.outer(v, v @ blk)


def apply_right(A, v, tau, rows, cols):
    """A[rows, cols] <- A[rows, cols] (I - tau v v^T)."""
    if tau == 0.0:
        return
    blk = A[rows, cols]
    A[rows, cols] = blk - tau * np.outer(blk @ v, v)


def hessenberg_reduce(A):
    """Householder reduction A = Q H Q^T with H upper Hessenberg (paper eq.
    ``hessenberg_form``, phase (i) of Sec. 1).  Unblocked textbook algorithm
    (Golub & Van Loan Alg. 7.4.2): for column j the reflector of
    A[j+1:, j] is applied from both sides and accumulated into Q.

    Returns (H, Q).  Entries below the first subdiagonal are set to 0.
    """
    H = np.array(A, dtype=np.float64, copy=True)
    n = H.shape[0]
    Q = np.eye(n)
    for j in range(n - 2):
        v, tau, beta = reflector(H[j + 1:, j])
        rows = slice(j + 1, n)
        apply_left(H, v, tau, rows, slice(j, n))
        apply_right(H, v, tau, slice(0, n), rows)
        apply_right(Q, v, tau, slice(0, n), rows)
        H[j + 1, j] = beta
        H[j + 2:, j] = 0.0
    return H, Q
