"""Accuracy metrics (paper Sec. 5.4), eigenvectors of a quasi-triangular Schur
factor and eigenvalue condition numbers (oracle).

Test infrastructure only (see ``oracle/__init__``).
"""

import numpy as np

from .qr import U, eig_from_schur


def r_a(A, X, Q):
    """R_A(X, Q) = ||Q X Q^T - A||_F / (u ||A||_F), eq. RsepA (Sec. 5.4)."""
    return np.linalg.norm(Q @ X @ Q.T - A) / (U * np.linalg.norm(A))


def r_orth(Q):
    """R_orth(Q) = ||Q Q^T - I||_F / (u ||I||_F), eq. Rorth (Sec. 5.4)."""
    n = Q.shape[0]
    return np.linalg.norm(Q @ Q.T - np.eye(n)) / (U * np.sqrt(n))


def e_lambda(computed, exact):
    """E_lambda of Sec. 5.4 for every computed eigenvalue:
    min over exact lambda of |computed - lambda| / (u |lambda|)."""
    exact = np.asarray(exact)
    return np.array([np.min(np.abs(c - exact) / (U * np.abs(exact))) for c in np.asarray(computed)])


def schur_structure_errors(S, tol=0.0):
    """List of violations of the standardised real Schur form (eq.
    ``2by2_blocks``): entries below the subdiagonal, two consecutive nonzero
    subdiagonals, 2x2 blocks with unequal diagonal or b*c >= 0."""
    n = S.shape[0]
    errs = []
    if n >= 3 and np.max(np.abs(np.tril(S, -2))) > tol:
        errs.append("below-subdiagonal entries")
    j = 0
    while j < n - 1:
        if S[j + 1, j] != 0.0:
            if j + 2 < n and S[j + 2, j + 1] != 0.0:
                errs.append(f"consecutive subdiagonals at {j}")
            if S[j, j] != S[j + 1, j + 1]:
                errs.append(f"unequal diagonal in 2x2 block at {j}")
            if S[j, j + 1] * S[j + 1, j] >= 0.0:
                errs.append(f"real 2x2 block at {j}")
            j += 2
        else:
            j += 1
    return errs


def _blocks(S):
    n = S.shape[0]
    out = []
    j = 0
    while j < n:
        if j + 1 < n and S[j + 1, j] != 0.0:
            out.append((j, 2))
            j += 2
        else:
            out.append((j, 1))
            j += 1
    return out


def _solve_shifted(B, lam, rhs, smin):
    """Solve (B - lam I) x = rhs for a 1x1 or 2x2 real block B and complex
    lam; a pivot below smin is replaced by smin (perturbation of a nearly
    repeated eigenvalue)."""
    if B.shape[0] == 1:
        d = B[0, 0] - lam
        if abs(d) < smin:
            d = smin
        return rhs / d
    M = B.astype(complex) - lam * np.eye(2)
    det = M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]
    if abs(det) < smin * max(1.0, np.max(np.abs(M))):
        det = smin * max(1.0, np.max(np.abs(M)))
    return np.array([M[1, 1] * rhs[0] - M[0, 1] * rhs[1], -M[1, 0] * rhs[0] + M[0, 0] * rhs[1]]) / det


def eigvecs_quasi_triangular(S):
    """Right eigenvectors X (S X = X diag(lam)) and vectors W with
    S^T W = W diag(lam), i.e. W = conj(Y) for left eigenvectors Y
    (y^H S = lam y^H), of a standardised quasi-triangular S, by block back
    (resp. forward) substitution; columns have unit 2-norm.

    Returns (lam, X, W), lam ordered as ``eig_from_schur``.
    """
    n = S.shape[0]
    wr, wi = eig_from_schur(S)
    lam = wr + 1j * wi
    blocks = _blocks(S)
    smin = max(U * np.linalg.norm(S), 1e-300)
    X = np.zeros((n, n), dtype=complex)
    W = np.zeros((n, n), dtype=complex)
    for bi, (s0, sz) in enumerate(blocks):
        for e in range(sz):
            i = s0 + e
            l = lam[i]
            x = np.zeros(n, dtype=complex)
            w = np.zeros(n, dtype=complex)
            end = s0 + sz
            if sz == 1:
                x[s0] = 1.0
                w[s0] = 1.0
            else:
                a, b, c, d = S[s0, s0], S[s0, s0 + 1], S[s0 + 1, s0], S[s0 + 1, s0 + 1]
                x[s0:end] = [b, l - a] if abs(b) + abs(l - a) > 0 else [l - d, c]
                w[s0:end] = [c, l - a] if abs(c) + abs(l - a) > 0 else [l - d, b]
            for (t0, tz) in reversed(blocks[:bi]):
                rhs = -S[t0:t0 + tz, t0 + tz:end] @ x[t0 + tz:end]
                x[t0:t0 + tz] = _solve_shifted(S[t0:t0 + tz, t0:t0 + tz], l, rhs, smin)
            for (t0, tz) in blocks[bi + 1:]:
                rhs = -S[s0:t0, t0:t0 + tz].T @ w[s0:t0]
                w[t0:t0 + tz] = _solve_shifted(S[t0:t0 + tz, t0:t0 + tz].T, l, rhs, smin)
            X[:, i] = x / np.linalg.norm(x)
            W[:, i] = w / np.linalg.norm(w)
    return lam, X, W


def eig_condition(S):
    """Eigenvalue condition numbers kappa_i = ||x_i|| ||y_i|| / |y_i^H x_i|
    (>= 1) of the quasi-triangular S (the same for H = Z S Z^T)."""
    lam, X, W = eigvecs_quasi_triangular(S)
    c = np.abs(np.sum(W * X, axis=0))
    return lam, 1.0 / np.maximum(c, 1e-300)


def match_eigenvalues(a, b):
    """Optimal one-to-one matching of two eigenvalue multisets (Hungarian
    assignment on |a_i - b_j|; scipy's linear_sum_assignment is used as a
    library primitive).  Returns (perm, dist) with b[perm[i]] matched to
    a[i]."""
    from scipy.optimize import linear_sum_assignment
    a = np.asarray(a)
    b = np.asarray(b)
    C = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(C)
    perm = np.empty(len(a), dtype=int)
    perm[r] = c
    return perm, C[r, c][np.argsort(r)]
