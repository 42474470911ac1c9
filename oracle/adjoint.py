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
