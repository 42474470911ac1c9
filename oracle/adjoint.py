"""Eigenvalue adjoint (oracle).  Test infrastructure only.

Not in the paper.  For a real loss L = sum_i f(lam_i) of the eigenvalues of
H, write g_i = df/dRe(lam_i) + i df/dIm(lam_i), so that a perturbation moves
L by Re(conj(g_i) dlam_i).  First-order perturbation theory gives
dlam_i = y_i^H dH x_i / (y_i^H x_i) for right / left eigenvectors
(H x = lam x, y^H H = lam y^H), hence

    dL/dH = Re( sum_i conj(g_i) / c_i * conj(y_i) x_i^T ),  c_i = y_i^H x_i.

With H = Z S Z^T and the eigenvectors of S (x = Z x_S, y = Z y_S) this is
Z G_S Z^T with G_S built from S alone; ``metrics.eigvecs_quasi_triangular``
returns w = conj(y_S), so G_S = Re(sum_i conj(g_i)/(w_i^T x_i) w_i x_i^T).
"""

import numpy as np

from .metrics import eigvecs_quasi_triangular


def eig_adjoint_schur(S, gwr, gwi):
    """G_S for cotangents (gwr, gwi) of the eigenvalues in the order of
    ``qr.eig_from_schur(S)``."""
    lam, X, W = eigvecs_quasi_triangular(S)
    g = np.asarray(gwr) + 1j * np.asarray(gwi)
    c = np.sum(W * X, axis=0)
    coef = np.conj(g) / c
    return np.real((W * coef[None, :]) @ X.T)


def eig_adjoint(S, Z, gwr, gwi):
    """dL/dH = Z G_S Z^T."""
    return Z @ eig_adjoint_schur(S, gwr, gwi) @ Z.T


# --------------------------------------------------- Schur-factor cotangents

def _block_of(S):
    n = S.shape[0]
    blk = np.zeros(n, dtype=int)
    starts = []
    j = 0
    while j < n:
        starts.append(j)
        if j + 1 < n and S[j + 1, j] != 0.0:
            blk[j] = blk[j + 1] = len(starts) - 1
            j += 2
        else:
            blk[j] = len(starts) - 1
            j += 1
    return blk, starts


def _schur_gauge_system(S):
    """The linear conditions that fix the first-order change of the real
    Schur factorisation H = Z S Z^T (not in the paper).  With dZ = Z Omega
    (Omega skew) and E = Z^T dH Z, the factor changes by
        dS = E + S Omega - Omega S;
    Omega's unknowns are its entries below the diagonal outside the 2x2
    diagonal blocks and the one inside each 2x2 block; the conditions are
    that dS stays zero below the diagonal blocks and that each 2x2 block stays
    standardised (equal diagonal entries: d(S_kk - S_k+1,k+1) = 0).

    Returns (unknowns, rows, M) with M the matrix of the conditions applied to
    S Omega - Omega S for each unknown's Omega = e_i e_j^T - e_j e_i^T, so
    that the unknowns l solve M l = -cond(E)."""
    n = S.shape[0]
    blk, starts = _block_of(S)
    unknowns = [(i, j) for i in range(n) for j in range(i) if blk[i] != blk[j]]
    pairs = [k for k in starts if k + 1 < n and blk[k + 1] == blk[k]]
    unknowns += [(k + 1, k) for k in pairs]
    rows = [("off", i, j) for (i, j) in unknowns if blk[i] != blk[j]] + [("blk", k, k) for k in pairs]

    def cond(D):
        return np.array([D[i, j] if kind == "off" else D[i, i] - D[i + 1, i + 1] for kind, i, j in rows])

    M = np.zeros((len(rows), len(unknowns)))
    for u, (i, j) in enumerate(unknowns):
        Om = np.zeros((n, n))
        Om[i, j] = 1.0
        Om[j, i] = -1.0
        M[:, u] = cond(S @ Om - Om @ S)
    return unknowns, rows, M, cond


def schur_tangent(S, Z, dH):
    """(dS, dZ) of the standardised real Schur factors for the perturbation
    dH, from the conditions of ``_schur_gauge_system`` (dense solve)."""
    n = S.shape[0]
    unknowns, rows, M, cond = _schur_gauge_system(S)
    E = Z.T @ dH @ Z
    l = -np.linalg.solve(M, cond(E)) if unknowns else np.zeros(0)
    Om = np.zeros((n, n))
    for v, (i, j) in zip(l, unknowns):
        Om[i, j] = v
        Om[j, i] = -v
    return E + S @ Om - Om @ S, Z @ Om


def schur_factor_adjoint(S, Z, Sbar, Zbar):
    """dL/dH for a loss L(S, Z) of the standardised real Schur factors with
    cotangents Sbar = dL/dS, Zbar = dL/dZ: the transpose of
    ``schur_tangent``.  With G = S^T Sbar - Sbar S^T + Z^T Zbar, the unknowns'
    cotangents are w_ij = G_ij - G_ji; y = -M^-T w; then
    Ebar = Sbar + (y placed on the condition rows' entries: E_ij for an
    off-block row, +E_kk and -E_k+1,k+1 for a block row) and
    dL/dH = Z Ebar Z^T."""
    unknowns, rows, M, cond = _schur_gauge_system(S)
    G = S.T @ Sbar - Sbar @ S.T + Z.T @ Zbar
    Ebar = np.array(Sbar, dtype=np.float64, copy=True)
    if unknowns:
        w = np.array([G[i, j] - G[j, i] for (i, j) in unknowns])
        y = -np.linalg.solve(M.T, w)
        for yr, (kind, i, j) in zip(y, rows):
            if kind == "off":
                Ebar[i, j] += yr
            else:
                Ebar[i, i] += yr
                Ebar[i + 1, i + 1] -= yr
    return Z @ Ebar @ Z.T
