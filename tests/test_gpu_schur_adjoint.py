"""Schur-factor adjoint on the GPU (schur_factor_backward) against the
oracle's dense adjoint on the same factors (entrywise, within
1e-10 * scale, scale = ||Sbar|| + ||Zbar|| times the conditioning of the
gauge system, bounded here by the inputs' eigenvalue separation), closed
forms that hold at any order (L = tr S, L = ||S||_F^2 give I and 2 H), and
finite differences of a sign-invariant loss through the GPU's own forward."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint, qr  # noqa: E402
from paper_2007_03576_gb300 import api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _np(T):
    return T.detach().cpu().numpy()


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (5, 3), (12, 4), (30, 5), (48, 6)])
def test_schur_factor_backward_matches_oracle(n, seed):
    H = inputs.hessrand(n, seed)
    S, Z, wr, wi, info = qr.schur(H)
    rng = np.random.default_rng(seed)
    Sb, Zb = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    ref = adjoint.schur_factor_adjoint(S, Z, Sb, Zb)
    got = _np(api.schur_factor_backward(_dev(S), _dev(Z), _dev(Sb), _dev(Zb)))
    assert np.max(np.abs(got - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [200, 1024])
def test_schur_factor_backward_closed_forms(n):
    """L = tr S = tr H -> I; L = ||S||_F^2 = ||H||_F^2 -> 2 H (the gauge
    terms must cancel exactly in both); L = ||Z||_F^2 = n -> 0."""
    H = inputs.hessrand(n, 900 + n)
    Hd = _dev(H)
    S, Z, wr, wi, info = api.schur(Hd)
    assert info == 0
    zero = torch.zeros_like(S)
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    g = api.schur_factor_backward(S, Z, eye, zero)
    assert float(torch.max(torch.abs(g - eye))) <= 1e-11
    g = api.schur_factor_backward(S, Z, 2 * S, zero)
    assert float(torch.max(torch.abs(g - 2 * Hd))) <= 1e-10 * float(torch.linalg.norm(Hd))
    g = api.schur_factor_backward(S, Z, zero, 2 * Z)
    assert float(torch.max(torch.abs(g))) <= 1e-11


def _fd_check(H, seed, h=1e-6):
    """Central-difference check of L = sum W * S^2 + sum V * Z^2 (blind to
    the signs of Z's columns) through api.schur_factors, along a Hessenberg
    direction; returns None when the factors are not smooth along the segment
    (a 2x2 block standardised on the other of its two branches, or another
    deflation order: |S| then moves by O(1) instead of O(h))."""
    n = H.shape[0]
    rng = np.random.default_rng(seed)
    Wt, Vt = _dev(rng.standard_normal((n, n))), _dev(rng.standard_normal((n, n)))
    dH = _dev(np.triu(rng.standard_normal((n, n)), -1))
    with torch.no_grad():
        S0, _ = api.schur_factors(_dev(H))
        Sp, Zp = api.schur_factors(_dev(H) + h * dH)
        Sm, Zm = api.schur_factors(_dev(H) - h * dH)
    moved = max(float(torch.max(torch.abs(Sp.abs() - S0.abs()))), float(torch.max(torch.abs(Sm.abs() - S0.abs()))))
    if moved > 1e-3:
        return None
    Hd = _dev(H).requires_grad_(True)
    S, Z = api.schur_factors(Hd)
    L = torch.sum(Wt * S * S) + torch.sum(Vt * Z * Z)
    L.backward()
    with torch.no_grad():
        Lp = torch.sum(Wt * Sp * Sp) + torch.sum(Vt * Zp * Zp)
        Lm = torch.sum(Wt * Sm * Sm) + torch.sum(Vt * Zm * Zm)
    return float((Lp - Lm) / (2 * h)), float(torch.sum(Hd.grad * dH))


def test_schur_factors_autograd_finite_differences_real_spectrum():
    """Non-normal matrices with a real spectrum (no 2x2 blocks, so the factors
    are smooth wherever the deflation order is kept); of a fixed list of
    seeds, those whose order is kept along the segment are checked (at least
    one must be)."""
    from oracle import householder
    n = 24
    checked = 0
    for seed in (90, 92, 94, 96):
        rng = np.random.default_rng(seed)
        T = 0.3 * np.triu(rng.uniform(-1, 1, (n, n)), 1) + np.diag(np.linspace(-3.0, 4.0, n))
        Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
        H = householder.hessenberg_reduce(Q @ T @ Q.T)[0]
        r = _fd_check(H, seed + 1)
        if r is None:
            continue
        fd, an = r
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (seed, fd, an)
        checked += 1
    assert checked >= 1


def test_schur_factors_autograd_finite_differences_complex_pairs():
    """hess_n matrices (complex pairs): the seeds of a fixed list whose factors
    stay on one branch along the segment are checked (at least one must)."""
    n = 24
    checked = 0
    for seed in range(77, 89):
        r = _fd_check(inputs.hessrand(n, seed), seed)
        if r is None:
            continue
        fd, an = r
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (seed, fd, an)
        checked += 1
    assert checked >= 1


def test_schur_factor_backward_batched_matches_single():
    sizes = [7, 64, 33, 150]
    Ss, Zs, Sbs, Zbs = [], [], [], []
    for i, n in enumerate(sizes):
        S, Z, wr, wi, info = api.schur(_dev(inputs.hessrand(n, 600 + i)))
        rng = np.random.default_rng(600 + i)
        Ss.append(S)
        Zs.append(Z)
        Sbs.append(_dev(rng.standard_normal((n, n))))
        Zbs.append(_dev(rng.standard_normal((n, n))))
    outs = api.schur_factor_backward_batched(Ss, Zs, Sbs, Zbs)
    for S, Z, Sb, Zb, g in zip(Ss, Zs, Sbs, Zbs, outs):
        assert torch.equal(g, api.schur_factor_backward(S, Z, Sb, Zb))
