"""The generalized case on the GPU (schur_qz, schur_qz_batched,
schur_qz_sweep) against the QZ oracle (oracle/qz.py).

One sweep with identical inputs and shifts applies the same reflectors in
the same order on both sides, so it is compared entrywise (within
1e-12 ||H||_F).  Whole reductions are compared on what is unique: the
eigenvalues as a multiset (within 1e-10 kappa_i (||H|| + |lambda_i| ||T||),
kappa_i from LAPACK's left/right vectors), the number of infinite
eigenvalues and their place at the top, and the properties any correct
result has: (Q S Z^T, Q T Z^T) = (H, T0) and orthogonality within
1e-13 (relative, / sqrt(n)), and the standardised generalized Schur
structure.
"""

import ctypes
import math

import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")

from oracle import metrics, qz  # noqa: E402
from paper_2007_03576_gb300 import _lib, api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _np(T):
    return T.detach().cpu().numpy()


def _check_pair(H0, T0, S, T, Q, Z, tol=1e-13):
    n = H0.shape[0]
    assert np.linalg.norm(Q @ S @ Z.T - H0) <= tol * np.linalg.norm(H0)
    assert np.linalg.norm(Q @ T @ Z.T - T0) <= tol * np.linalg.norm(T0)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * math.sqrt(n)
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= tol * math.sqrt(n)
    assert qz.gschur_structure_errors(S, T) == []


def _eig_close(lam, H0, T0, tol=1e-10):
    """Finite eigenvalues against LAPACK's, scaled by their condition."""
    w, vl, vr = scipy.linalg.eig(H0, T0, left=True, right=True)
    fin = np.isfinite(w) & (np.abs(w) < 1e12)
    w, vl, vr = w[fin], vl[:, fin], vr[:, fin]
    kap = np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0) / np.abs(np.sum(np.conj(vl) * (T0 @ vr), axis=0))
    mine = lam[np.isfinite(lam)]
    assert len(mine) == len(w)
    perm, dist = metrics.match_eigenvalues(w, mine)
    scale = kap * (np.linalg.norm(H0) + np.abs(w) * np.linalg.norm(T0))
    assert np.all(dist <= tol * scale), float(np.max(dist / scale))


@pytest.mark.parametrize("n,lo,hi", [(3, 0, 2), (9, 0, 8), (40, 5, 33), (130, 0, 129)])
def test_qz_sweep_matches_oracle(n, lo, hi):
    H, T = inputs.ht_pair(n, 100 + n)
    ssum, sprod = 0.3, 1.7
    Ho, To, Qo, Zo = H.copy(), T.copy(), np.eye(n), np.eye(n)
    qz.qz_sweep(Ho, To, Qo, Zo, lo, hi, ssum, sprod)
    Hd, Td, Qd, Zd = _dev(H), _dev(T), _dev(np.eye(n)), _dev(np.eye(n))
    api.qz_sweep(Hd, Td, Qd, Zd, lo, hi, ssum, sprod)
    nh = np.linalg.norm(H)
    assert np.max(np.abs(_np(Hd) - Ho)) <= 1e-12 * nh
    assert np.max(np.abs(_np(Td) - To)) <= 1e-12 * np.linalg.norm(T)
    assert np.max(np.abs(_np(Qd) - Qo)) <= 1e-12
    assert np.max(np.abs(_np(Zd) - Zo)) <= 1e-12


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (17, 4), (64, 5), (100, 6), (201, 7)])
def test_qz_matches_oracle(n, seed):
    H, T = inputs.ht_pair(n, seed)
    S, Tt, Q, Z, ar, ai, be, info = api.qz(_dev(H), _dev(T))
    assert info == 0
    Sg, Tg, Qg, Zg = _np(S), _np(Tt), _np(Q), _np(Z)
    _check_pair(H, T, Sg, Tg, Qg, Zg)
    lam = qz.eigenvalues(_np(ar), _np(ai), _np(be))
    So, To, Qo, Zo, aro, aio, beo, info_o = qz.qz(H, T)
    assert info_o == 0
    lo_ = qz.eigenvalues(aro, aio, beo)
    perm, dist = metrics.match_eigenvalues(lo_, lam)
    assert np.max(dist) <= 1e-10 * max(1.0, np.max(np.abs(lo_)))
    if n > 2:
        _eig_close(lam, H, T)
    # beta >= 0 for real eigenvalues, complex pairs positive imaginary part first
    bg = _np(be)
    assert np.all(bg >= 0.0)


@pytest.mark.parametrize("n,nsing", [(12, 1), (30, 3), (80, 5)])
def test_qz_infinite_eigenvalues(n, nsing):
    """T with nsing zero diagonal entries: as many infinite eigenvalues as
    LAPACK counts (adjacent zeros can merge, so the count is LAPACK's, not
    nsing) and as the oracle finds, chased to the top (T's leading diagonal
    entries zero)."""
    H, T = inputs.ht_pair(n, 300 + n, singular=nsing)
    w, b = scipy.linalg.eigvals(H, T, homogeneous_eigvals=True)
    ninf = int(np.sum(np.abs(b) <= 1e-12 * np.abs(w)))
    assert 1 <= ninf <= nsing
    S, Tt, Q, Z, ar, ai, be, info = api.qz(_dev(H), _dev(T))
    assert info == 0
    bg = _np(be)
    assert int(np.sum(bg == 0.0)) == ninf
    Tg = _np(Tt)
    assert np.all(np.diag(Tg)[:ninf] == 0.0)
    _check_pair(H, T, _np(S), Tg, _np(Q), _np(Z))
    So, To, Qo, Zo, aro, aio, beo, info_o = qz.qz(H, T)
    assert int(np.sum(beo == 0.0)) == ninf
    lam = qz.eigenvalues(_np(ar), _np(ai), bg)
    lo_ = qz.eigenvalues(aro, aio, beo)
    perm, dist = metrics.match_eigenvalues(lo_[np.isfinite(lo_)], lam[np.isfinite(lam)])
    assert np.max(dist) <= 1e-9 * max(1.0, np.max(np.abs(lo_[np.isfinite(lo_)])))


def test_qz_identity_t_and_accumulation():
    """T = I: the eigenvalues are H's (the standard QR path's); with Q1, Z1
    given they are multiplied in place (z_init = 1)."""
    n = 60
    H = inputs.hessrand(n, 41)
    S, Tt, Q, Z, ar, ai, be, info = api.qz(_dev(H), _dev(np.eye(n)))
    assert info == 0
    Sq, Zq, wr, wi, rc = api.schur(_dev(H))
    perm, dist = metrics.match_eigenvalues(_np(wr) + 1j * _np(wi), qz.eigenvalues(_np(ar), _np(ai), _np(be)))
    assert np.max(dist) <= 1e-11 * np.linalg.norm(H)
    rng = np.random.default_rng(5)
    Q1 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Z1 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    H2, T2 = inputs.ht_pair(n, 42)
    S, Tt, Q, Z, ar, ai, be, info = api.qz(_dev(H2), _dev(T2), _dev(Q1), _dev(Z1))
    assert info == 0
    assert np.linalg.norm(_np(Q) @ _np(S) @ _np(Z).T - Q1 @ H2 @ Z1.T) <= 1e-13 * np.linalg.norm(H2)


def test_qz_from_a_dense_pair():
    """A dense pair reduced to Hessenberg-triangular form by the oracle, then
    the GPU's QZ accumulating the reduction's Q1, Z1: (A, B) = Q (S, T) Z^T."""
    n = 90
    rng = np.random.default_rng(77)
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    H, R, Q1, Z1 = qz.hessenberg_triangular(A, B)
    S, Tt, Q, Z, ar, ai, be, info = api.qz(_dev(H), _dev(R), _dev(Q1), _dev(Z1))
    assert info == 0
    _check_pair(A, B, _np(S), _np(Tt), _np(Q), _np(Z))
    _eig_close(qz.eigenvalues(_np(ar), _np(ai), _np(be)), A, B)


def test_qz_batched_matches_single():
    sizes = [5, 33, 64, 17, 100, 3]
    pairs = [inputs.ht_pair(n, 500 + i, singular=(1 if i == 2 else 0)) for i, n in enumerate(sizes)]
    Hs = [_dev(H) for H, _ in pairs]
    Ts = [_dev(T) for _, T in pairs]
    Qs = [api.new_colmajor(n) for n in sizes]
    Zs = [api.new_colmajor(n) for n in sizes]
    ars = [torch.empty(n, dtype=torch.float64, device="cuda") for n in sizes]
    ais = [torch.empty_like(a) for a in ars]
    bes = [torch.empty_like(a) for a in ars]
    info = api.qz_batched_inplace(Hs, Ts, Qs, Zs, ars, ais, bes)
    assert info == [0] * len(sizes)
    for i, (H, T) in enumerate(pairs):
        _check_pair(H, T, _np(Hs[i]), _np(Ts[i]), _np(Qs[i]), _np(Zs[i]))
        S1, T1, Q1, Z1, a1, b1, c1, rc = api.qz(_dev(H), _dev(T))
        assert torch.equal(S1, Hs[i]) and torch.equal(T1, Ts[i]) and torch.equal(c1, bes[i])


def test_qz_edge_cases():
    # non-finite input: SCHUR_ERR_NONFINITE, pair unchanged
    H, T = inputs.ht_pair(10, 9)
    T[3, 5] = np.inf
    Hd, Td = _dev(H), _dev(T)
    Hc, Tc = Hd.clone(), Td.clone()
    lib = _lib.load()
    n = 10
    Q, Z = api.new_colmajor(n), api.new_colmajor(n)
    ar, ai, be = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream)
    rc = lib.schur_qz(n, Hd.data_ptr(), n, Td.data_ptr(), n, Q.data_ptr(), n, Z.data_ptr(), n, ar.data_ptr(),
                      ai.data_ptr(), be.data_ptr(), ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_NONFINITE
    assert torch.equal(Hd, Hc) and torch.equal(torch.nan_to_num(Td, posinf=1.0), torch.nan_to_num(Tc, posinf=1.0))
    # n = 0 and want_qz = False
    assert lib.schur_qz(0, None, 1, None, 1, None, 1, None, 1, None, None, None, None) == 0
    H, T = inputs.ht_pair(40, 10)
    S1, T1, _, _, a1, b1, c1, _ = api.qz(_dev(H), _dev(T))
    S2, T2, Q2, Z2, a2, b2, c2, _ = api.qz(_dev(H), _dev(T), want_qz=False)
    assert Q2 is None and torch.equal(S1, S2) and torch.equal(c1, c2)
    # an all-zero T: every eigenvalue infinite
    n = 8
    H = inputs.hessrand(n, 11)
    S, Tt, Q, Z, ar, ai, be, info = api.qz(_dev(H), _dev(np.zeros((n, n))))
    assert info == 0 and np.all(_np(be) == 0.0)
    _check_pair(H, np.zeros((n, n)), _np(S), _np(Tt), _np(Q), _np(Z))
