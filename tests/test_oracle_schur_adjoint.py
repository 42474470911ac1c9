"""Pins of the oracle's Schur-factor tangent and adjoint (oracle/adjoint.py:
schur_tangent, schur_factor_adjoint) against finite differences of the
oracle's own Schur form, the transpose identity between the two, and closed
forms: L = tr S and L = ||S||_F^2 are functions of H alone (tr H, ||H||_F^2),
so their gradients are I and 2 H whatever the gauge terms do."""

import numpy as np
import pytest

from oracle import adjoint, qr
from paper_2007_03576_gb300 import inputs


def _sign_fix(S, Z, Zref):
    s = np.sign(np.sum(Z * Zref, axis=0))
    return S * np.outer(s, s), Z * s


@pytest.mark.parametrize("n,seed", [(4, 1), (9, 2), (14, 3), (21, 5)])
def test_schur_tangent_matches_finite_differences(n, seed):
    H = inputs.hessrand(n, seed)
    S, Z, wr, wi, info = qr.schur(H)
    rng = np.random.default_rng(seed)
    dH = np.triu(rng.standard_normal((n, n)), -1)
    dS, dZ = adjoint.schur_tangent(S, Z, dH)
    h = 1e-6
    Sp, Zp, wrp, _, _ = qr.schur(H + h * dH)
    Sm, Zm, wrm, _, _ = qr.schur(H - h * dH)
    # differences are meaningful only along the same deflation order
    assert np.max(np.abs(wrp - wr)) <= 1e-4 and np.max(np.abs(wrm - wr)) <= 1e-4
    Sp, Zp = _sign_fix(Sp, Zp, Z)
    Sm, Zm = _sign_fix(Sm, Zm, Z)
    scale = max(1.0, np.max(np.abs(dS)))
    assert np.max(np.abs((Sp - Sm) / (2 * h) - dS)) <= 1e-6 * scale
    assert np.max(np.abs((Zp - Zm) / (2 * h) - dZ)) <= 1e-6 * scale
    # the tangent keeps the structure: zero below the blocks, equal diagonals in 2x2 blocks
    for k in range(n - 1):
        if S[k + 1, k] != 0.0:
            assert abs(dS[k, k] - dS[k + 1, k + 1]) <= 1e-12 * scale
    low = np.tril(np.ones((n, n), dtype=bool), -2)
    assert np.max(np.abs(dS[low])) <= 1e-12 * scale


@pytest.mark.parametrize("n,seed", [(5, 11), (12, 12), (30, 13)])
def test_schur_adjoint_is_the_transpose_of_the_tangent(n, seed):
    H = inputs.hessrand(n, seed)
    S, Z, wr, wi, info = qr.schur(H)
    rng = np.random.default_rng(seed)
    Sb, Zb = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    Hb = adjoint.schur_factor_adjoint(S, Z, Sb, Zb)
    for _ in range(3):
        dH = rng.standard_normal((n, n))
        dS, dZ = adjoint.schur_tangent(S, Z, dH)
        lhs = np.sum(Hb * dH)
        rhs = np.sum(Sb * dS) + np.sum(Zb * dZ)
        assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + np.linalg.norm(Hb) * np.linalg.norm(dH))


def test_schur_adjoint_closed_forms():
    n = 16
    H = inputs.hessrand(n, 21)
    S, Z, wr, wi, info = qr.schur(H)
    zero = np.zeros((n, n))
    assert np.max(np.abs(adjoint.schur_factor_adjoint(S, Z, np.eye(n), zero) - np.eye(n))) <= 1e-12
    assert np.max(np.abs(adjoint.schur_factor_adjoint(S, Z, 2 * S, zero) - 2 * H)) <= 1e-11 * np.linalg.norm(H)
    # ||Z||_F^2 = n: no dependence on H
    assert np.max(np.abs(adjoint.schur_factor_adjoint(S, Z, zero, 2 * Z))) <= 1e-12


def test_schur_adjoint_loss_gradient_by_finite_differences():
    """A loss invariant under the sign choice of Z's columns:
    L = sum W * S^2 + sum V * Z^2, gradient vs central differences."""
    n = 10
    H = inputs.hessrand(n, 31)
    rng = np.random.default_rng(31)
    Wt, Vt = rng.standard_normal((n, n)), rng.standard_normal((n, n))

    def loss(Hx):
        S, Z, *_ = qr.schur(Hx)
        return np.sum(Wt * S * S) + np.sum(Vt * Z * Z)

    S, Z, *_ = qr.schur(H)
    Hb = adjoint.schur_factor_adjoint(S, Z, 2 * Wt * S, 2 * Vt * Z)
    dH = np.triu(rng.standard_normal((n, n)), -1)
    h = 1e-6
    fd = (loss(H + h * dH) - loss(H - h * dH)) / (2 * h)
    assert abs(fd - np.sum(Hb * dH)) <= 1e-6 * max(1.0, abs(fd))
