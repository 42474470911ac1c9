"""Hessenberg-triangular reduction on the GPU (schur_ht_reduce,
schur_ht_reduce_batched) against the oracle's reduction (oracle/qz.py,
hessenberg_triangular).

Both apply the same reflectors and rotations in the same order, so the
reduced pair and both transformations are compared entrywise: within
1e-11 ||A||_F (H), 1e-11 ||B||_F (R) and 1e-11 (Q, Z).  Larger pairs are
checked on what any correct reduction satisfies: (A, B) = Q (H, R) Z^T and
orthogonality within 1e-13 (relative, / sqrt(n)), exact zeros below H's
subdiagonal and R's diagonal; and the whole generalized pipeline on the GPU
(reduction, then QZ) against LAPACK's generalized eigenvalues.
"""

import ctypes
import math

import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")

from oracle import metrics, qz  # noqa: E402
from paper_2007_03576_gb300 import _lib, api  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _np(T):
    return T.detach().cpu().numpy()


def _pair(n, seed):
    rng = np.random.default_rng([seed, 13])
    return rng.standard_normal((n, n)), rng.standard_normal((n, n))


def _check_props(A, B, H, R, Q, Z, tol=1e-13):
    n = A.shape[0]
    assert np.all(np.tril(H, -2) == 0.0) and np.all(np.tril(R, -1) == 0.0)
    assert np.linalg.norm(Q @ H @ Z.T - A) <= tol * math.sqrt(n) * np.linalg.norm(A)
    assert np.linalg.norm(Q @ R @ Z.T - B) <= tol * math.sqrt(n) * np.linalg.norm(B)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= tol * math.sqrt(n)
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= tol * math.sqrt(n)


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (8, 4), (33, 5), (100, 6), (257, 7), (400, 8)])
def test_ht_matches_oracle(n, seed):
    A, B = _pair(n, seed)
    Ho, Ro, Qo, Zo = qz.hessenberg_triangular(A, B)
    H, R, Q, Z = api.ht_reduce(_dev(A), _dev(B))
    H, R, Q, Z = _np(H), _np(R), _np(Q), _np(Z)
    assert np.max(np.abs(H - Ho)) <= 1e-11 * np.linalg.norm(A)
    assert np.max(np.abs(R - Ro)) <= 1e-11 * np.linalg.norm(B)
    assert np.max(np.abs(Q - Qo)) <= 1e-11
    assert np.max(np.abs(Z - Zo)) <= 1e-11
    _check_props(A, B, H, R, Q, Z)


def test_ht_large_pair_properties_and_no_qz():
    """Order 700 (1024-thread blocks): the factorisation properties; with
    want_qz off, the same (H, R)."""
    n = 700
    A, B = _pair(n, 70)
    H, R, Q, Z = api.ht_reduce(_dev(A), _dev(B))
    _check_props(A, B, _np(H), _np(R), _np(Q), _np(Z))
    H2, R2, Q2, Z2 = api.ht_reduce(_dev(A), _dev(B), want_qz=False)
    assert Q2 is None and torch.equal(H, H2) and torch.equal(R, R2)


def test_ht_accumulates_into_given_q_z():
    n = 50
    A, B = _pair(n, 80)
    rng = np.random.default_rng(81)
    Q0 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Z0 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    H, R, Q, Z = api.ht_reduce(_dev(A), _dev(B), _dev(Q0), _dev(Z0))
    H1, R1, Q1, Z1 = api.ht_reduce(_dev(A), _dev(B))
    assert torch.equal(H, H1) and torch.equal(R, R1)
    assert np.max(np.abs(_np(Q) - Q0 @ _np(Q1))) <= 1e-13 * n
    assert np.max(np.abs(_np(Z) - Z0 @ _np(Z1))) <= 1e-13 * n


def test_ht_batched_matches_single():
    sizes = [5, 64, 17, 130, 3, 1, 2]
    pairs = [_pair(n, 90 + i) for i, n in enumerate(sizes)]
    As = [_dev(a) for a, _ in pairs]
    Bs = [_dev(b) for _, b in pairs]
    Qs = [api.new_colmajor(n) for n in sizes]
    Zs = [api.new_colmajor(n) for n in sizes]
    info = api.ht_reduce_batched_inplace(As, Bs, Qs, Zs)
    assert info == [0] * len(sizes)
    for (a, b), H, R, Q, Z in zip(pairs, As, Bs, Qs, Zs):
        H1, R1, Q1, Z1 = api.ht_reduce(_dev(a), _dev(b))
        assert torch.equal(H, H1) and torch.equal(R, R1) and torch.equal(Q, Q1) and torch.equal(Z, Z1)


def test_ht_special_pairs():
    """B already triangular (stage 1 reflectors are the identity), B = 0
    (both stages leave B zero), A already Hessenberg with B = I (no
    rotation moves anything: H = A, R = I, Q = Z = I)."""
    n = 40
    A, B = _pair(n, 100)
    Bt = np.triu(B)
    H, R, Q, Z = api.ht_reduce(_dev(A), _dev(Bt))
    Ho, Ro, Qo, Zo = qz.hessenberg_triangular(A, Bt)
    assert np.max(np.abs(_np(H) - Ho)) <= 1e-11 * np.linalg.norm(A)
    _check_props(A, Bt, _np(H), _np(R), _np(Q), _np(Z))
    H, R, Q, Z = api.ht_reduce(_dev(A), _dev(np.zeros((n, n))))
    assert np.all(_np(R) == 0.0)
    _check_props(A, np.zeros((n, n)), _np(H), _np(R), _np(Q), _np(Z))
    Ah = np.triu(A, -1)
    H, R, Q, Z = api.ht_reduce(_dev(Ah), _dev(np.eye(n)))
    assert np.array_equal(_np(H), Ah) and np.array_equal(_np(R), np.eye(n))
    assert np.array_equal(_np(Q), np.eye(n)) and np.array_equal(_np(Z), np.eye(n))


def test_ht_nonfinite_input_unchanged():
    n = 12
    A, B = _pair(n, 110)
    B[4, 7] = np.nan
    Ad, Bd = _dev(A), _dev(B)
    Ac, Bc = Ad.clone(), Bd.clone()
    Q, Z = api.new_colmajor(n), api.new_colmajor(n)
    lib = _lib.load()
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream)
    rc = lib.schur_ht_reduce(n, Ad.data_ptr(), n, Bd.data_ptr(), n, Q.data_ptr(), n, Z.data_ptr(), n,
                             ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_NONFINITE
    assert torch.equal(Ad, Ac) and torch.equal(torch.nan_to_num(Bd), torch.nan_to_num(Bc))
    assert lib.schur_ht_reduce(0, None, 1, None, 1, None, 1, None, 1, None) == 0


@pytest.mark.parametrize("n,seed", [(60, 120), (200, 121)])
def test_generalized_pipeline_on_gpu(n, seed):
    """Dense pair -> GPU reduction -> GPU QZ: (A, B) = Q (S, T) Z^T and the
    eigenvalues within 1e-10 kappa_i (||A|| + |lambda_i| ||B||) of LAPACK's
    (scipy), kappa_i from LAPACK's left and right vectors."""
    A, B = _pair(n, seed)
    S, T, Q, Z, ar, ai, be, info = api.generalized_schur(_dev(A), _dev(B))
    assert info == 0
    Sg, Tg, Qg, Zg = _np(S), _np(T), _np(Q), _np(Z)
    assert np.linalg.norm(Qg @ Sg @ Zg.T - A) <= 1e-13 * math.sqrt(n) * np.linalg.norm(A)
    assert np.linalg.norm(Qg @ Tg @ Zg.T - B) <= 1e-13 * math.sqrt(n) * np.linalg.norm(B)
    assert qz.gschur_structure_errors(Sg, Tg) == []
    lam = qz.eigenvalues(_np(ar), _np(ai), _np(be))
    w, vl, vr = scipy.linalg.eig(A, B, left=True, right=True)
    kap = np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0) / np.abs(np.sum(np.conj(vl) * (B @ vr), axis=0))
    perm, dist = metrics.match_eigenvalues(w, lam)
    scale = kap * (np.linalg.norm(A) + np.abs(w) * np.linalg.norm(B))
    assert np.all(dist <= 1e-10 * scale), float(np.max(dist / scale))
