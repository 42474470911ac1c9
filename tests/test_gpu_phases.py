"""The phases around the QR iteration on the GPU, through the C ABI: the
Householder reduction A = Q H Q^T before it and the eigenvectors from the
Schur form after it (Sec. 1, phases (i) and (iii)).

Parity with the oracle.  The reduction uses the oracle's reflector
convention (LAPACK's), so the same input gives the same H and Q up to
rounding: compared entrywise within 1e-12 ||A||_F at orders the oracle
finishes in seconds.  Eigenvectors are unique up to a complex scale; both
sides fix it the same way (1 on a 1x1 block, (b, lambda - a) on a 2x2 block,
then unit 2-norm), so they are compared entrywise as well, within
1e-11 ||S||_F / gap_i (first-order perturbation of an eigenvector, gap_i the
distance from lambda_i to the nearest other eigenvalue; rounding is
~n u ||S||_F).  At the 4096 workload size, properties that hold at any size:
backward error and orthogonality (<= 1e-13, the paper's Sec. 5.4 metrics),
entries fixed exactly by the algorithm, eigen-residuals, bit-reproducible
reruns.
"""

import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import householder, metrics, qr  # noqa: E402
from paper_2007_03576_gb300 import _lib, api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _np(T):
    return T.detach().cpu().numpy()


# ------------------------------------------------------------ reduction


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (5, 4), (64, 5), (100, 6), (257, 7), (300, 8)])
def test_hessenberg_reduce_matches_oracle(n, seed):
    A = inputs.gaussian(n, seed)
    Ho, Qo = householder.hessenberg_reduce(A)
    H, Q = api.hessenberg_reduce(_dev(A))
    Hg, Qg = _np(H), _np(Q)
    nA = np.linalg.norm(A)
    assert np.all(np.tril(Hg, -2) == 0.0)
    assert np.max(np.abs(Hg - Ho)) <= 1e-12 * nA
    assert np.max(np.abs(Qg - Qo)) <= 1e-12
    st = api.last_stats()
    assert st["flops"] == pytest.approx(sum(8.0 * m * m + 4.0 * n * m for m in range(2, n)) if n > 2 else 0.0)


def test_hessenberg_reduce_special_inputs():
    n = 150
    rng = np.random.default_rng(11)
    # already upper Hessenberg: every reflector is the identity, H = A and Q = I exactly
    A = np.triu(rng.standard_normal((n, n)), -1)
    H, Q = api.hessenberg_reduce(_dev(A))
    assert np.array_equal(_np(H), A)
    assert np.array_equal(_np(Q), np.eye(n))
    # zero tails in some columns (identity reflectors in the middle of the reduction)
    A = rng.standard_normal((n, n))
    A[5:, 3] = 0.0
    A[40:, 30] = 0.0
    A[n - 3:, n - 5] = 0.0
    Ho, Qo = householder.hessenberg_reduce(A)
    H, Q = api.hessenberg_reduce(_dev(A))
    assert np.max(np.abs(_np(H) - Ho)) <= 1e-12 * np.linalg.norm(A)
    assert np.max(np.abs(_np(Q) - Qo)) <= 1e-12
    # scale invariance near the ends of the exponent range (the norm is taken
    # from the column scaled by its largest entry there); powers of two scale exactly
    A = inputs.gaussian(n, 12)
    H1, Q1 = api.hessenberg_reduce(_dev(A))
    for e in (600, -600):
        c = 2.0 ** e
        H2, Q2 = api.hessenberg_reduce(_dev(A * c))
        assert np.max(np.abs(_np(H2) / c - _np(H1))) <= 1e-13 * np.linalg.norm(A)
        assert np.max(np.abs(_np(Q2) - _np(Q1))) <= 1e-13
    # Q not wanted: the same H, bit for bit
    H3, Q3 = api.hessenberg_reduce(_dev(A), want_q=False)
    assert Q3 is None and torch.equal(H3, H1)


def test_hessenberg_reduce_rejects_nonfinite():
    A = inputs.gaussian(40, 13)
    A[17, 3] = np.nan
    Ad = _dev(A)
    before = Ad.clone()
    lib = _lib.load()
    Q = api.new_colmajor(40)
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream)
    rc = lib.schur_hessenberg_reduce(40, Ad.data_ptr(), 40, Q.data_ptr(), 40, ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_NONFINITE
    assert torch.equal(torch.nan_to_num(Ad, nan=7.0), torch.nan_to_num(before, nan=7.0))


def test_hessenberg_reduce_n4096():
    """The n = 4096 workload size: a seeded dense N(0,1) matrix."""
    n = 4096
    A = inputs.gaussian(n, 2022)
    Ad = _dev(A)
    H, Q = api.hessenberg_reduce(Ad)
    torch.cuda.synchronize()
    nA = torch.linalg.norm(Ad)
    ra = float(torch.linalg.norm(Q @ H @ Q.T - Ad) / nA)
    ro = float(torch.linalg.norm(Q.T @ Q - torch.eye(n, dtype=torch.float64, device="cuda")) / math.sqrt(n))
    assert ra <= 1e-13, ra
    assert ro <= 1e-13, ro
    assert float(torch.max(torch.abs(torch.tril(H, -2)))) == 0.0
    # entries the algorithm fixes exactly: row/column 0 of Q, H[0, 0], |H[1, 0]|
    Qn = _np(Q)
    e0 = np.zeros(n)
    e0[0] = 1.0
    assert np.array_equal(Qn[:, 0], e0) and np.array_equal(Qn[0, :], e0)
    Hn = _np(H)
    assert Hn[0, 0] == A[0, 0]
    assert abs(abs(Hn[1, 0]) - np.linalg.norm(A[1:, 0])) <= 1e-14 * np.linalg.norm(A[1:, 0])
    assert np.sign(Hn[1, 0]) == -np.sign(A[1, 0])
    # bit-reproducible (no atomics): a rerun gives the same H and Q
    H2, Q2 = api.hessenberg_reduce(Ad)
    assert torch.equal(H, H2) and torch.equal(Q, Q2)


# ---------------------------------------------------------- eigenvectors


def _oracle_vectors(S, Z):
    lam, X, W = metrics.eigvecs_quasi_triangular(S)
    return lam, (Z @ X if Z is not None else X)


def _gaps(lam):
    d = np.abs(lam[:, None] - lam[None, :])
    np.fill_diagonal(d, np.inf)
    return np.min(d, axis=1) if lam.size > 1 else np.array([np.inf])


def _compare(Xg, Xo, lam, nS):
    tol = 1e-11 * nS / np.minimum(_gaps(lam), nS)
    err = np.max(np.abs(Xg - Xo), axis=0)
    assert np.all(err <= tol), float(np.max(err / tol))


@pytest.mark.parametrize("n,seed", [(1, 21), (2, 22), (7, 23), (64, 24), (65, 25), (130, 26), (200, 27)])
def test_eigenvectors_match_oracle(n, seed):
    H = inputs.hessrand(n, seed)
    S, Z, wr, wi, info = qr.schur(H)
    assert info == 0
    lam, Xo = _oracle_vectors(S, Z)
    wrd, wid = torch.from_numpy(wr).cuda(), torch.from_numpy(wi).cuda()
    X = api.eigenvectors(_dev(S), _dev(Z), wrd, wid)
    Xg = _np(api.complex_eigenvectors(X, wid))
    _compare(Xg, Xo, lam, np.linalg.norm(S))
    assert np.allclose(np.linalg.norm(Xg, axis=0), 1.0, atol=1e-14)
    # eigen-residual of H itself
    assert np.max(np.abs(H @ Xg - Xg * lam[None, :])) <= 1e-12 * np.linalg.norm(H)
    # without Z: the eigenvectors of S
    lam, Xs = _oracle_vectors(S, None)
    Xg = _np(api.complex_eigenvectors(api.eigenvectors(_dev(S), None, wrd, wid), wid))
    _compare(Xg, Xs, lam, np.linalg.norm(S))


def test_eigenvectors_special_cases():
    # diagonal S: the unit vectors, exactly
    n = 70
    d = np.arange(1.0, n + 1.0)
    S = np.diag(d)
    X = api.eigenvectors(_dev(S), None, torch.from_numpy(d).cuda(), torch.zeros(n, dtype=torch.float64).cuda())
    assert np.array_equal(_np(X), np.eye(n))
    # one standardised 2x2 block [[a, b], [c, a]] (bc < 0): x = (b, i sqrt(-bc)) / norm
    a, b, c = 0.5, 2.0, -0.5
    S = np.array([[a, b], [c, a]])
    w = math.sqrt(-b * c)
    X = api.eigenvectors(_dev(S), None, torch.tensor([a, a], dtype=torch.float64).cuda(),
                         torch.tensor([w, -w], dtype=torch.float64).cuda())
    x = np.array([b, 1j * w]) / math.hypot(b, w)
    Xn = _np(X)
    assert np.allclose(Xn[:, 0] + 1j * Xn[:, 1], x, atol=1e-15)
    # repeated eigenvalue (a Jordan block): the perturbed pivot gives a finite unit vector, as in the oracle
    S = np.array([[1.0, 1.0, 0.3], [0.0, 1.0, 2.0], [0.0, 0.0, 1.0]])
    lam, Xo = _oracle_vectors(S, None)
    X = api.eigenvectors(_dev(S), None, torch.ones(3, dtype=torch.float64).cuda(),
                         torch.zeros(3, dtype=torch.float64).cuda())
    Xg = _np(X)
    assert np.all(np.isfinite(Xg))
    assert np.allclose(np.linalg.norm(Xg, axis=0), 1.0, atol=1e-14)
    assert np.max(np.abs(Xg - Xo.real)) <= 1e-12


@pytest.mark.parametrize("n,seed", [(300, 31), (1000, 32)])
def test_eig_pipeline_general_matrix(n, seed):
    """Every phase on the GPU for a dense matrix: reduction, Schur form
    accumulating the reduction's Q, eigenvectors carried back."""
    A = inputs.gaussian(n, seed)
    wr, wi, X, info = api.eig(_dev(A))
    assert info == 0
    lam = _np(wr) + 1j * _np(wi)
    Xg = _np(api.complex_eigenvectors(X, wi))
    assert np.max(np.abs(A @ Xg - Xg * lam[None, :])) <= 1e-12 * np.linalg.norm(A)
    assert np.allclose(np.linalg.norm(Xg, axis=0), 1.0, atol=1e-13)
    import scipy.linalg
    w, vl, vr = scipy.linalg.eig(A, left=True, right=True)
    kap = 1.0 / np.abs(np.sum(np.conj(vl) * vr, axis=0))
    perm, dist = metrics.match_eigenvalues(w, lam)
    assert np.all(dist <= 1e-10 * kap * np.linalg.norm(A))


def test_eigenvectors_n4096_pipeline():
    """At the n = 4096 workload size: eigen-residual of every vector of the
    Hessenberg matrix through the GPU path, and unit norms."""
    n = 4096
    H = inputs.hessrand(n, 2021)
    Hd = _dev(H)
    S, Z, wr, wi, info = api.schur(Hd)
    assert info == 0
    X = api.eigenvectors(S, Z, wr, wi)
    Xc = api.complex_eigenvectors(X, wi)
    lam = torch.complex(wr, wi)
    R = Hd.to(torch.complex128) @ Xc - Xc * lam[None, :]
    res = float(torch.max(torch.abs(R)) / torch.linalg.norm(Hd))
    assert res <= 1e-12, res
    nrm = torch.linalg.norm(Xc, dim=0)
    assert float(torch.max(torch.abs(nrm - 1.0))) <= 1e-13
