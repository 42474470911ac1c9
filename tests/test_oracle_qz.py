"""Pins of the QZ oracle (oracle/qz.py) against what the mathematics fixes:
library runs of LAPACK's generalized eigensolver (scipy), pencils with a
known spectrum built from their generalized Schur form, the implicit-Q
property of one sweep, the B = I case (the standard QR iteration), and
infinite eigenvalues of a singular B."""

import numpy as np
import pytest
import scipy.linalg

from oracle import metrics, qr, qz


def _pencil(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n)), rng.standard_normal((n, n))


def _haar(n, rng):
    Qm, Rm = np.linalg.qr(rng.standard_normal((n, n)))
    return Qm * np.sign(np.diag(Rm))[None, :]


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (8, 3), (31, 4)])
def test_hessenberg_triangular_reduction(n, seed):
    A, B = _pencil(n, seed)
    H, R, Q, Z = qz.hessenberg_triangular(A, B)
    assert np.all(np.tril(H, -2) == 0.0) and np.all(np.tril(R, -1) == 0.0)
    assert np.linalg.norm(Q @ H @ Z.T - A) <= 1e-14 * n * np.linalg.norm(A)
    assert np.linalg.norm(Q @ R @ Z.T - B) <= 1e-14 * n * np.linalg.norm(B)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-14 * n
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= 1e-14 * n
    # the pair keeps its generalized eigenvalues (library run of LAPACK)
    perm, dist = metrics.match_eigenvalues(scipy.linalg.eigvals(H, R), scipy.linalg.eigvals(A, B))
    assert np.max(dist) <= 1e-9 * max(1.0, np.max(np.abs(scipy.linalg.eigvals(A, B))))


@pytest.mark.parametrize("n,seed", [(3, 11), (6, 12), (25, 13), (60, 14)])
def test_qz_matches_lapack_eigenvalues(n, seed):
    A, B = _pencil(n, seed)
    H, R, Q1, Z1 = qz.hessenberg_triangular(A, B)
    S, T, Q, Z, ar, ai, be, info = qz.qz(H, R, Q1, Z1)
    assert info == 0
    assert qz.gschur_structure_errors(S, T) == []
    assert np.linalg.norm(Q @ S @ Z.T - A) <= 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(Q @ T @ Z.T - B) <= 1e-13 * np.linalg.norm(B)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * np.sqrt(n)
    lam = qz.eigenvalues(ar, ai, be)
    ref = scipy.linalg.eigvals(A, B)
    # condition of each eigenvalue of the pencil from LAPACK's left/right vectors
    w, vl, vr = scipy.linalg.eig(A, B, left=True, right=True)
    kap = np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0) / np.abs(np.sum(np.conj(vl) * (B @ vr), axis=0))
    perm, dist = metrics.match_eigenvalues(ref, lam)
    scale = kap * (np.linalg.norm(A) + np.abs(ref) * np.linalg.norm(B))
    assert np.all(dist <= 1e-12 * scale)


def test_known_spectrum_pencil():
    """(A, B) = Qa (S0, T0) Za^T with S0, T0 upper triangular: eigenvalues
    S0_ii / T0_ii (closed form), including two complex pairs built as 2x2
    blocks of S0 with T0's block the identity."""
    rng = np.random.default_rng(21)
    n = 12
    S0 = np.triu(rng.uniform(-1, 1, (n, n)))
    T0 = np.triu(rng.uniform(-1, 1, (n, n)))
    d = np.array([1.0, -2.0, 3.0, 0.5, 4.0, -1.5, 2.5, -3.5, 0.0, 0.0, 0.0, 0.0])
    td = np.array([1.0, 2.0, 0.5, 1.0, 2.0, 1.0, 1.0, 0.25, 1.0, 1.0, 1.0, 1.0])
    np.fill_diagonal(S0, d)
    np.fill_diagonal(T0, td)
    known = list(d[:8] / td[:8])
    for k, (a, b) in zip((8, 10), ((1.0, 2.0), (-0.5, 0.75))):
        S0[k:k + 2, k:k + 2] = [[a, b], [-b, a]]
        T0[k:k + 2, k:k + 2] = np.eye(2)
        known += [complex(a, b), complex(a, -b)]
    Qa, Za = _haar(n, rng), _haar(n, rng)
    A, B = Qa @ S0 @ Za.T, Qa @ T0 @ Za.T
    H, R, Q1, Z1 = qz.hessenberg_triangular(A, B)
    S, T, Q, Z, ar, ai, be, info = qz.qz(H, R, Q1, Z1)
    assert info == 0
    perm, dist = metrics.match_eigenvalues(np.array(known), qz.eigenvalues(ar, ai, be))
    assert np.max(dist) <= 1e-11


def test_identity_b_is_the_qr_iteration():
    """B = I: the pair's eigenvalues are H's, as the standard QR iteration
    (the oracle's own, pinned separately) computes them."""
    rng = np.random.default_rng(31)
    n = 30
    A = rng.standard_normal((n, n))
    H, R, Q1, Z1 = qz.hessenberg_triangular(A, np.eye(n))
    assert np.linalg.norm(R - np.eye(n)) <= 1e-13
    S, T, Q, Z, ar, ai, be, info = qz.qz(H, R, Q1, Z1)
    Ss, Zs, wr, wi, info2 = qr.schur(H)
    perm, dist = metrics.match_eigenvalues(wr + 1j * wi, qz.eigenvalues(ar, ai, be))
    assert np.max(dist) <= 1e-12 * np.linalg.norm(A)


def test_one_sweep_implicit_q():
    """After one double-shift sweep the first column of Q is parallel to
    (M - l1)(M - l2) e1 with M = H T^-1 formed densely (the implicit-Q
    theorem behind Sec. 2.2's remark), and the pair is Hessenberg-triangular
    again and equivalent to the input."""
    rng = np.random.default_rng(41)
    n = 9
    H = np.triu(rng.standard_normal((n, n)), -1)
    T = np.triu(rng.standard_normal((n, n))) + 3.0 * np.eye(n)
    ssum, sprod = 0.7, 1.9
    M = H @ np.linalg.inv(T)
    p = (M @ M - ssum * M + sprod * np.eye(n))[:, 0]
    H2, T2 = H.copy(), T.copy()
    Q, Z = np.eye(n), np.eye(n)
    qz.qz_sweep(H2, T2, Q, Z, 0, n - 1, ssum, sprod)
    q1 = Q[:, 0]
    assert abs(abs(q1 @ p) - np.linalg.norm(p)) <= 1e-13 * np.linalg.norm(p)
    assert np.max(np.abs(np.tril(H2, -2))) == 0.0 and np.max(np.abs(np.tril(T2, -1))) == 0.0
    assert np.linalg.norm(Q @ H2 @ Z.T - H) <= 1e-13 * np.linalg.norm(H)
    assert np.linalg.norm(Q @ T2 @ Z.T - T) <= 1e-13 * np.linalg.norm(T)


def test_infinite_eigenvalues_chased_to_the_top():
    """A singular B of rank n - 2 gives exactly two infinite eigenvalues
    (beta = 0), deflated at the upper-left corner (Sec. 3.4: chased up the
    diagonal); the finite ones are LAPACK's."""
    rng = np.random.default_rng(51)
    n = 14
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    B[:, 4] = 0.0
    B[:, 9] = 2.0 * B[:, 2]
    H, R, Q1, Z1 = qz.hessenberg_triangular(A, B)
    S, T, Q, Z, ar, ai, be, info = qz.qz(H, R, Q1, Z1)
    assert info == 0
    assert int(np.sum(be == 0.0)) == 2
    assert T[0, 0] == 0.0 and T[1, 1] == 0.0
    assert np.linalg.norm(Q @ S @ Z.T - A) <= 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(Q @ T @ Z.T - B) <= 1e-13 * np.linalg.norm(B)
    lam = qz.eigenvalues(ar, ai, be)
    fin = lam[np.isfinite(lam)]
    ref = scipy.linalg.eigvals(A, B)
    ref = ref[np.isfinite(ref) & (np.abs(ref) < 1e8)]
    assert len(ref) == n - 2
    perm, dist = metrics.match_eigenvalues(ref, fin)
    assert np.max(dist) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("seed", range(6))
def test_standardize_pair_block(seed):
    """2x2 pair closed forms: complex eigenvalues keep their values with T's
    block diagonal and positive; real ones split S's block to triangular with
    the eigenvalues S_kk / T_kk."""
    rng = np.random.default_rng(60 + seed)
    S2 = rng.standard_normal((2, 2))
    T2 = np.triu(rng.standard_normal((2, 2))) + np.diag([2.0, 2.0])
    lam, cpx = qz.pair_eigs_2x2(S2, T2)
    ref = scipy.linalg.eigvals(S2, T2)
    perm, dist = metrics.match_eigenvalues(ref, lam)
    assert np.max(dist) <= 1e-13 * np.max(np.abs(ref))
    S, T, Q, Z = S2.copy(), T2.copy(), np.eye(2), np.eye(2)
    was_cpx = qz.standardize_pair_block(S, T, Q, Z, 0)
    assert was_cpx == cpx
    assert np.linalg.norm(Q @ S @ Z.T - S2) <= 1e-14 * 10 and np.linalg.norm(Q @ T @ Z.T - T2) <= 1e-14 * 10
    if cpx:
        assert T[0, 1] == 0.0 and T[0, 0] > 0 and T[1, 1] > 0
    else:
        assert S[1, 0] == 0.0 and T[1, 0] == 0.0
        perm, dist = metrics.match_eigenvalues(ref, np.array([S[0, 0] / T[0, 0], S[1, 1] / T[1, 1]]))
        assert np.max(dist) <= 1e-12 * np.max(np.abs(ref))


def test_ht_subdiag_negligible_boundaries():
    """The QZ deflation test on H: an entry just at u (|h_{k-1,k-1}| +
    |h_kk|) is negligible, one ulp-scale step above it is not; the sum uses
    both diagonal entries (swapping one for its neighbour moves the
    boundary); with zero diagonal entries the smlnum floor decides."""
    from oracle.qr import U, smlnum

    n = 6
    H = np.triu(np.ones((n, n)), -1)
    H[2, 2], H[3, 3] = 3.0, 5.0
    thr = U * (3.0 + 5.0)
    H[3, 2] = thr
    assert qz.ht_subdiag_negligible(H, 3, n)
    H[3, 2] = thr * (1.0 + 4 * U)
    assert not qz.ht_subdiag_negligible(H, 3, n)
    H[3, 2] = U * (3.0 + 1.0) * 1.5        # above u (|h22| + |h23|) but below the true threshold
    assert qz.ht_subdiag_negligible(H, 3, n)
    H[2, 2] = H[3, 3] = 0.0
    H[3, 2] = smlnum(n)
    assert qz.ht_subdiag_negligible(H, 3, n)
    H[3, 2] = 2.0 * smlnum(n)
    assert not qz.ht_subdiag_negligible(H, 3, n)


@pytest.mark.parametrize("seed", range(4))
def test_trailing_shift_pair_against_dense_m(seed):
    """(ssum, sprod) = trace and determinant of the trailing 2x2 of
    M = H T^-1 formed with the dense inverse of the whole T (the routine uses
    only a 3x3 window of T); T = I reduces it to H's trailing 2x2."""
    rng = np.random.default_rng(70 + seed)
    n = 9
    H = np.triu(rng.standard_normal((n, n)), -1)
    T = np.triu(rng.standard_normal((n, n))) + 3.0 * np.eye(n)
    for lo, hi in [(0, n - 1), (2, 6), (4, 6)]:
        M = H @ np.linalg.inv(T)
        m = M[hi - 1:hi + 1, hi - 1:hi + 1]
        ssum, sprod = qz.trailing_shift_pair(H, T, lo, hi)
        assert abs(ssum - np.trace(m)) <= 1e-12 * np.abs(m).sum()
        assert abs(sprod - np.linalg.det(m)) <= 1e-12 * np.abs(m).sum() ** 2
    ssum, sprod = qz.trailing_shift_pair(H, np.eye(n), 0, n - 1)
    h = H[n - 2:, n - 2:]
    assert abs(ssum - np.trace(h)) <= 1e-14 * np.abs(h).sum()
    assert abs(sprod - np.linalg.det(h)) <= 1e-13 * np.abs(h).sum() ** 2


def test_exceptional_shift_pair_with_identity_t_is_the_qr_one():
    """T = I: the generalized exceptional pair equals the standard QR
    iteration's (EISPACK's constants, pinned with the n-cycle matrix)."""
    rng = np.random.default_rng(80)
    n = 8
    H = np.triu(rng.standard_normal((n, n)), -1)
    for lo, hi in [(0, n - 1), (3, 6), (5, 6)]:
        got = qz.exceptional_shift_pair(H, np.eye(n), lo, hi)
        want = qr.exceptional_pairs(H, lo, hi, 1)[0]
        assert np.allclose(got, want, rtol=1e-15, atol=0.0)
