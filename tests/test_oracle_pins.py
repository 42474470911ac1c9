"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, characteristic polynomials, matrices with known spectra,
invariants, the implicit-Q theorem and library routines on the same input.

Each test names the part of the oracle it pins and the passage of the paper
(Myllykoski, ACM TOMS 2021) that defines it.
"""

import math

import numpy as np
import pytest
import scipy.linalg

from oracle import householder, qr, metrics, adjoint, testmats
from deflation_cases import SML4, SUBDIAG_CASES, SPIKE_CASES, spike_case_args
from paper_2007_03576_gb300 import inputs

U = qr.U


def _eig_close(computed, exact, tol):
    perm, dist = metrics.match_eigenvalues(np.asarray(computed), np.asarray(exact))
    assert np.max(dist) <= tol, (np.max(dist), tol)


def _check_schur(H, S, Z, tol_ra=1e-13, tol_orth=None):
    n = H.shape[0]
    ra = np.linalg.norm(Z @ S @ Z.T - H) / np.linalg.norm(H)
    ro = np.linalg.norm(Z.T @ Z - np.eye(n)) / math.sqrt(n)
    assert ra <= tol_ra, ra
    assert ro <= (tol_orth if tol_orth is not None else 1e-13), ro
    assert metrics.schur_structure_errors(S) == []


# ---------------------------------------------------------------- reflectors


def test_reflector_maps_to_e1():
    """Householder reflector (Sec. 2.2 footnote: Q^T v is a multiple of e_1)."""
    rng = np.random.default_rng(1)
    for m in (2, 3, 7):
        x = rng.standard_normal(m)
        v, tau, beta = householder.reflector(x)
        P = np.eye(m) - tau * np.outer(v, v)
        assert np.allclose(P @ P.T, np.eye(m), atol=1e-15)
        y = P @ x
        assert abs(y[0] - beta) < 1e-14 * np.linalg.norm(x)
        assert np.max(np.abs(y[1:])) < 1e-14 * np.linalg.norm(x)
        assert abs(abs(beta) - np.linalg.norm(x)) < 1e-14 * np.linalg.norm(x)
    v, tau, beta = householder.reflector(np.array([3.0, 0.0, 0.0]))
    assert tau == 0.0 and beta == 3.0


def test_hessenberg_reduction_matches_lapack():
    """Phase (i) (Sec. 1): same Householder convention as LAPACK dgehrd, so
    scipy.linalg.hessenberg (a library run) gives the same H up to rounding."""
    A = inputs.gaussian(60, 3)
    H, Q = householder.hessenberg_reduce(A)
    Hs, Qs = scipy.linalg.hessenberg(A, calc_q=True)
    assert np.max(np.abs(np.tril(H, -2))) == 0.0
    assert np.linalg.norm(Q @ H @ Q.T - A) < 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(60)) < 1e-13
    # signs of the reflectors agree with LAPACK's, so H matches entrywise
    assert np.max(np.abs(H - Hs)) < 1e-12 * np.linalg.norm(A)


# ---------------------------------------------------------------- 2x2 blocks


@pytest.mark.parametrize("seed", range(20))
def test_standardize_2x2_closed_form(seed):
    """P1: eigenvalues (a+d)/2 +- sqrt(((a-d)/2)^2 + bc) and the standard form
    of eq. 2by2_blocks (equal diagonal, bc < 0 for complex; c = 0 for real)."""
    rng = np.random.default_rng(seed)
    a, b, c, d = rng.standard_normal(4) * rng.uniform(0.1, 10)
    if seed % 5 == 0:
        c = 0.0
    disc = ((a - d) / 2) ** 2 + b * c
    cs, sn, B = qr.standardize_2x2(a, b, c, d)
    G = np.array([[cs, -sn], [sn, cs]])
    A = np.array([[a, b], [c, d]])
    assert abs(cs * cs + sn * sn - 1) < 1e-15
    assert np.max(np.abs(G.T @ A @ G - B)) < 1e-14 * np.max(np.abs(A))
    if disc >= 0:
        assert B[1, 0] == 0.0
        got = sorted([B[0, 0], B[1, 1]])
        r = math.sqrt(disc)
        exp = sorted([(a + d) / 2 - r, (a + d) / 2 + r])
        assert np.allclose(got, exp, atol=1e-13 * np.max(np.abs(A)))
    else:
        assert B[0, 0] == B[1, 1] and B[0, 1] * B[1, 0] < 0
        assert abs(B[0, 0] - (a + d) / 2) < 1e-14 * np.max(np.abs(A))
        assert abs(math.sqrt(-B[0, 1] * B[1, 0]) - math.sqrt(-disc)) < 1e-13 * np.max(np.abs(A))


def test_schur_2x2_and_trivial():
    """n = 1, 2 and a zero subdiagonal through the full driver."""
    S, Z, wr, wi, info = qr.schur(np.array([[3.0]]))
    assert info == 0 and wr[0] == 3.0 and Z[0, 0] == 1.0
    for H in (np.array([[1.0, 2.0], [-3.0, 1.5]]), np.array([[1.0, 2.0], [0.0, -4.0]]),
              np.array([[0.0, 1.0], [1.0, 0.0]])):
        S, Z, wr, wi, info = qr.schur(H)
        a, b, c, d = H.ravel()
        ref = np.linalg.eigvals(H)
        _eig_close(wr + 1j * wi, ref, 1e-14 * 4)
        _check_schur(H, S, Z)


# ------------------------------------------------------- brute force n <= 4


def _charpoly(H):
    """Characteristic polynomial coefficients by the Faddeev-LeVerrier
    recursion (exact algebra, independent of any eigensolver)."""
    n = H.shape[0]
    c = [1.0]
    M = np.zeros_like(H)
    for k in range(1, n + 1):
        M = H @ M + c[-1] * np.eye(n)
        c.append(-np.trace(H @ M) / k)
    return np.array(c)


@pytest.mark.parametrize("n", [3, 4])
@pytest.mark.parametrize("seed", range(6))
def test_brute_force_small(n, seed):
    """P2: roots of det(lambda I - H) (Faddeev-LeVerrier coefficients, roots
    by numpy.roots) equal the oracle's eigenvalues; det(lambda I - H) ~ 0 at
    each computed eigenvalue."""
    H = inputs.hessrand(n, 100 + seed)
    c = _charpoly(H)
    S, Z, wr, wi, info = qr.schur(H)
    lam = wr + 1j * wi
    _eig_close(lam, np.roots(c), 1e-11 * np.linalg.norm(H))
    for l in lam:
        assert abs(np.linalg.det(l * np.eye(n) - H)) <= 1e-10 * np.linalg.norm(H) ** n
    _check_schur(H, S, Z)


# ------------------------------------------------------- known spectra


@pytest.mark.parametrize("roots", [
    [1, -1, 2, -2, 3, -3, 4],
    [0.5, 1.5, 2.5, -1 + 2j, -1 - 2j, 3j, -3j, 2 + 1j, 2 - 1j],
    list(np.exp(2j * np.pi * np.arange(8) / 8) * 1.5) + [0.25, -0.25],
])
def test_companion_known_roots(roots):
    """P3: companion matrix of a polynomial with prescribed well-separated
    roots."""
    H = testmats.companion(roots)
    S, Z, wr, wi, info = qr.schur(H)
    assert info == 0
    _eig_close(wr + 1j * wi, roots, 1e-8 * max(1, np.max(np.abs(roots))))
    _check_schur(H, S, Z, tol_ra=1e-13)


@pytest.mark.parametrize("n", [4, 9, 16, 31, 64])
def test_cyclic_roots_of_unity(n):
    """P3: the n-cycle permutation (eigenvalues exp(2 pi i k / n)); standard
    shifts stall on it, so this exercises the exceptional shifts."""
    H = testmats.cyclic(n)
    P = qr.Params(nmin=12, nwin_francis=12) if n >= 31 else qr.Params()
    S, Z, wr, wi, info = qr.schur(H, params=P)
    assert info == 0
    _eig_close(wr + 1j * wi, np.exp(2j * np.pi * np.arange(n) / n), 1e-12)
    _check_schur(H, S, Z)


@pytest.mark.parametrize("nonnormal", [False, True])
def test_prescribed_spectrum(nonnormal):
    """P4: orthogonally similar to a prescribed block-diagonal matrix (the
    n = 4096 workload's second family, at n = 96)."""
    H, lam = testmats.prescribed(96, np.random.default_rng(7), nonnormal)
    S, Z, wr, wi, info = qr.schur(H, params=qr.Params(nmin=20))
    assert info == 0
    kap_lam, kap = metrics.eig_condition(S)
    perm, dist = metrics.match_eigenvalues(wr + 1j * wi, lam)
    assert np.all(dist <= 100 * U * np.linalg.norm(H) * kap), np.max(dist / kap)
    _check_schur(H, S, Z)


def test_syn_family():
    """syn_n of Sec. 5.3: known eigenvalues +-1, +-3, ... half lifted to
    complex pairs r +- i|r|; E_lambda small (Sec. 5.4)."""
    H, lam = testmats.syn(64, np.random.default_rng(2020))
    assert np.sum(np.abs(lam.imag) > 0) == 32
    S, Z, wr, wi, info = qr.schur(H, params=qr.Params(nmin=16))
    assert info == 0
    e = metrics.e_lambda(wr + 1j * wi, lam)
    assert np.max(e) < 1e5, np.max(e)
    _check_schur(H, S, Z)


# ------------------------------------------------------- invariants / library


@pytest.mark.parametrize("n,nmin", [(40, 75), (90, 75), (120, 16)])
def test_invariants_and_scipy(n, nmin):
    """P5 / P6: sum(lambda) = tr H, sum(lambda^2) = tr H^2, residual and
    orthogonality of Sec. 5.4, and the eigenvalue multiset of LAPACK dgeev
    (scipy.linalg.eigvals, a library run) on the same hess_n input."""
    H = inputs.hessrand(n, 11 + n)
    S, Z, wr, wi, info = qr.schur(H, params=qr.Params(nmin=nmin))
    assert info == 0
    lam = wr + 1j * wi
    nh = np.linalg.norm(H)
    assert abs(np.sum(lam) - np.trace(H)) < 1e-12 * n * nh
    assert abs(np.sum(lam ** 2) - np.trace(H @ H)) < 1e-12 * n * nh ** 2
    _check_schur(H, S, Z, tol_ra=1e-13)
    _, kap = metrics.eig_condition(S)
    perm, dist = metrics.match_eigenvalues(lam, scipy.linalg.eigvals(H))
    assert np.all(dist <= 1e3 * U * nh * kap), np.max(dist / (U * nh * kap))


# ------------------------------------------------------- implicit Q theorem


def _poly_qr_step(H, shifts):
    """Explicit shifted QR step: p(H) = prod (H - s_i I) = Q R, H' = Q^T H Q."""
    n = H.shape[0]
    M = np.eye(n, dtype=complex)
    for s in shifts:
        M = M @ (H - s * np.eye(n))
    Q, R = np.linalg.qr(np.real(M))
    return Q.T @ H @ Q, Q


@pytest.mark.parametrize("shifts", [
    [0.3 + 1.1j, 0.3 - 1.1j],
    [0.5, -0.7],
    [0.2 + 0.4j, 0.2 - 0.4j, -1.0, 1.3],
    [0.9, 0.1, -0.5 + 0.5j, -0.5 - 0.5j, 2.0, -2.0],
])
def test_sweep_implicit_q(shifts):
    """Implicit-Q theorem (Sec. 2.2): a Francis / multishift sweep with shifts
    s_1..s_k equals the explicit QR step on p(H) = prod (H - s_i I), up to the
    signs of Q's columns.  Pins the bulge introduction vector, the chase
    geometry and the bottom-to-top pipelining of Sec. 2.3."""
    n = 14
    H = inputs.hessrand(n, 42) / math.sqrt(n)
    Hp, Q = _poly_qr_step(H, shifts)
    pairs = []
    i = 0
    while i < len(shifts):
        s1, s2 = shifts[i], shifts[i + 1]
        pairs.append(((s1 + s2).real, (s1 * s2).real))
        i += 2
    Hs = H.copy()
    Zs = np.eye(n)
    qr.multishift_sweep(Hs, Zs, 0, n - 1, pairs)
    D = np.sign(np.diag(Zs.T @ Q))
    assert np.all(D != 0)
    assert np.max(np.abs(Zs * D[None, :] - Q)) < 1e-10
    assert np.max(np.abs(D[:, None] * Hs * D[None, :] - Hp)) < 1e-10
    assert np.max(np.abs(np.tril(Hs, -2))) < 1e-12


# ------------------------------------------------------- reordering


def _quasi_tri(sizes, rng):
    n = sum(sizes)
    T = np.triu(rng.standard_normal((n, n)), 1)
    j = 0
    lams = []
    for s in sizes:
        if s == 1:
            T[j, j] = rng.uniform(-3, 3)
            lams.append([T[j, j]])
        else:
            a, b, c = rng.uniform(-3, 3), rng.uniform(0.5, 2), -rng.uniform(0.5, 2)
            T[j:j + 2, j:j + 2] = [[a, b], [c, a]]
            lams.append([a + 1j * math.sqrt(-b * c), a - 1j * math.sqrt(-b * c)])
        j += s
    return T, lams


@pytest.mark.parametrize("p,q", [(1, 1), (1, 2), (2, 1), (2, 2)])
@pytest.mark.parametrize("seed", range(4))
def test_swap_adjacent(p, q, seed):
    """Eigenvalue reordering (Sec. 2.5 step 2, Bai & Demmel direct swap): the
    blocks trade places (eigenvalues checked against the closed-form 2x2
    values), the similarity is orthogonal and the result stays standardised
    quasi-triangular."""
    rng = np.random.default_rng(seed)
    T, lams = _quasi_tri([1, p, q, 2], rng)
    T0 = T.copy()
    V = np.eye(T.shape[0])
    assert qr.swap_adjacent(T, V, 1, p, q)
    assert np.linalg.norm(V @ T @ V.T - T0) < 1e-13 * np.linalg.norm(T0)
    assert np.linalg.norm(V.T @ V - np.eye(T.shape[0])) < 1e-14
    assert metrics.schur_structure_errors(T) == []
    lead = np.linalg.eigvals(T[1:1 + q, 1:1 + q]) if q == 2 else [T[1, 1]]
    trail = np.linalg.eigvals(T[1 + q:1 + q + p, 1 + q:1 + q + p]) if p == 2 else [T[1 + q, 1 + q]]
    _eig_close(lead, lams[2], 1e-12)
    _eig_close(trail, lams[1], 1e-12)


def test_move_block_up():
    rng = np.random.default_rng(9)
    T, lams = _quasi_tri([1, 2, 1, 1, 2, 1, 2], rng)
    T0 = T.copy()
    V = np.eye(T.shape[0])
    assert qr.move_block_up(T, V, 8, 1)
    assert np.linalg.norm(V @ T @ V.T - T0) < 1e-13 * np.linalg.norm(T0)
    _eig_close(np.linalg.eigvals(T[1:3, 1:3]), lams[6], 1e-12)
    assert metrics.schur_structure_errors(T) == []


# ------------------------------------------------------- deflation / AED


def test_spike_test_thresholds():
    """Deflation conditions of Sec. 5.6 at their boundary (LAPACK-style,
    norm-stable, fixed)."""
    T = np.array([[2.0, 1.0, 0.0], [0.0, 1.0, 4.0], [0.0, -1.0, 1.0]])
    P = qr.Params()
    assert qr.spike_deflatable(T, np.array([0.5 * U * 2.0, 0, 0]), 0, 1, P, 3)
    assert not qr.spike_deflatable(T, np.array([2.0 * U * 2.0, 0, 0]), 0, 1, P, 3)
    hhat = 1.0 + 2.0   # sqrt|1*1| + sqrt|4*1|
    assert qr.spike_deflatable(T, np.array([0, 0.9 * U * hhat, 0.5 * U * hhat]), 2, 2, P, 3)
    assert not qr.spike_deflatable(T, np.array([0, 1.1 * U * hhat, 0.0]), 2, 2, P, 3)
    Pn = qr.Params(deflation="norm", normH=10.0)
    assert qr.spike_deflatable(T, np.array([9 * U, 0, 0]), 0, 1, Pn, 3)
    assert not qr.spike_deflatable(T, np.array([11 * U, 0, 0]), 0, 1, Pn, 3)
    Pf = qr.Params(deflation="fixed", thold=1e-3)
    assert qr.spike_deflatable(T, np.array([0, 9e-4, 9e-4]), 2, 2, Pf, 3)
    assert not qr.spike_deflatable(T, np.array([0, 9e-4, 2e-3]), 2, 2, Pf, 3)


def test_aed_decoupled_window_deflates_everything():
    """With a zero spike (h_{kwtop,kwtop-1} = 0) every candidate satisfies the
    deflation condition: AED returns nd = nw and the window in Schur form."""
    n, nw = 40, 12
    H = inputs.hessrand(n, 5)
    H[n - nw, n - nw - 1] = 0.0
    H0 = H.copy()
    Z = np.eye(n)
    nd, cands = qr.aed(H, Z, 0, n - 1, nw, qr.Params(normH=np.linalg.norm(H)))
    assert nd == nw and cands == []
    assert np.linalg.norm(Z @ H @ Z.T - H0) < 1e-13 * np.linalg.norm(H0)
    assert metrics.schur_structure_errors(H[n - nw:, n - nw:]) == []
    _eig_close(np.linalg.eigvals(H[n - nw:, n - nw:]), np.linalg.eigvals(H0[n - nw:, n - nw:]), 1e-11)


@pytest.mark.parametrize("seed", range(3))
def test_aed_step_properties(seed):
    """One AED step (Sec. 2.5): orthogonal similarity, Hessenberg form
    restored, deflated rows decoupled and in Schur form, and every deflated
    eigenvalue is an eigenvalue of H up to the size of the dropped spike
    entries (first-order perturbation times the condition number)."""
    n, nw = 80, 30
    H = inputs.hessrand(n, 300 + seed)
    # make the bottom converge: a few sweeps first
    Z = np.eye(n)
    P = qr.Params(normH=np.linalg.norm(H))
    for _ in range(3):
        qr.multishift_sweep(H, Z, 0, n - 1, [(0.0, 1.0), (1.0, 2.0)])
    H0 = H.copy()
    Z0 = Z.copy()
    nd, cands = qr.aed(H, Z, 0, n - 1, nw, P)
    assert np.linalg.norm(Z @ H @ Z.T - Z0 @ H0 @ Z0.T) < 1e-13 * np.linalg.norm(H0)
    assert np.max(np.abs(np.tril(H, -2))) == 0.0
    assert len(cands) == nw - nd
    if nd:
        k = n - nd
        assert H[k, k - 1] == 0.0
        Sd = H[k:, k:]
        assert metrics.schur_structure_errors(Sd) == []
        full = np.linalg.eigvals(H0)
        _eig_close(np.linalg.eigvals(Sd), full, 1e-8 * np.linalg.norm(H0))


def test_aed_recursive_window():
    """AED window larger than nmin: the window is reduced by the recursive
    multishift driver (Sec. 2.5 step 1, "recursive application of the QR
    algorithm")."""
    n = 120
    H = inputs.hessrand(n, 77)
    S, Z, wr, wi, info = qr.schur(H, params=qr.Params(nmin=12, nwin_francis=12, ns=6, nw=40))
    assert info == 0
    _check_schur(H, S, Z)
    _eig_close(wr + 1j * wi, scipy.linalg.eigvals(H), 1e-9 * np.linalg.norm(H))


@pytest.mark.parametrize("mode", ["norm", "fixed"])
def test_other_deflation_modes(mode):
    """Norm-stable and fixed deflation conditions (Sec. 5.6 items 2 and 3)."""
    H = inputs.hessrand(100, 8)
    P = qr.Params(deflation=mode, thold=1e-14 * np.linalg.norm(H), nmin=20)
    S, Z, wr, wi, info = qr.schur(H, params=P)
    assert info == 0
    _check_schur(H, S, Z)
    _eig_close(wr + 1j * wi, scipy.linalg.eigvals(H), 1e-9 * np.linalg.norm(H))


# ------------------------------------------------------- eigenvectors, adjoint


def test_eigvecs_quasi_triangular_vs_scipy():
    """Eigenvectors of S by block back-substitution: residuals, and condition
    numbers equal to those from scipy.linalg.eig (library run)."""
    H = inputs.hessrand(50, 4)
    S, Z, wr, wi, info = qr.schur(H)
    lam, X, W = metrics.eigvecs_quasi_triangular(S)
    assert np.max(np.abs(S @ X - X * lam[None, :])) < 1e-12 * np.linalg.norm(S)
    assert np.max(np.abs(S.T @ W - W * lam[None, :])) < 1e-12 * np.linalg.norm(S)
    _, kap = metrics.eig_condition(S)
    w, vl, vr = scipy.linalg.eig(S, left=True, right=True)
    kref = 1.0 / np.abs(np.sum(np.conj(vl) * vr, axis=0))
    perm, dist = metrics.match_eigenvalues(lam, w)
    assert np.allclose(kap, kref[perm], rtol=1e-6)


def test_adjoint_closed_forms():
    """P9: g = 1 for every eigenvalue gives dH = I (sum lambda = tr H);
    g = 2 conj(lambda) (L = sum Re lambda^2 = tr H^2) gives dH = 2 H^T."""
    H = inputs.hessrand(30, 6)
    S, Z, wr, wi, info = qr.schur(H)
    n = H.shape[0]
    dH = adjoint.eig_adjoint(S, Z, np.ones(n), np.zeros(n))
    assert np.max(np.abs(dH - np.eye(n))) < 1e-10
    dH = adjoint.eig_adjoint(S, Z, 2 * wr, -2 * wi)
    assert np.max(np.abs(dH - 2 * H.T)) < 1e-9 * np.linalg.norm(H)


def test_adjoint_finite_difference():
    """P9: L = sum |lambda|^2 (the differentiation workload's loss), central
    differences at h = 1e-6 along random Hessenberg-pattern directions."""
    n = 24
    H = inputs.hessrand(n, 13)
    S, Z, wr, wi, info = qr.schur(H)
    dH = adjoint.eig_adjoint(S, Z, 2 * wr, 2 * wi)

    def L(M):
        _, _, a, b, _ = qr.schur(M)
        return np.sum(a * a + b * b)

    rng = np.random.default_rng(0)
    for _ in range(3):
        E = np.triu(rng.standard_normal((n, n)), -1)
        h = 1e-6
        fd = (L(H + h * E) - L(H - h * E)) / (2 * h)
        an = np.sum(dH * E)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_syn_base_spectrum_golden():
    """Sec. 5.3 item 2: the base spectrum +-1, +-3, ... of syn_n (stored
    fixture) and the lifting rule r -> r +- i|r| for the paired entries."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "syn_spectrum_n8.txt")
    base = np.loadtxt(path)
    H, lam = testmats.syn(8, np.random.default_rng(1))
    reals = sorted(l.real for l in lam)
    # every lifted pair shares the real part of its first member
    for l in lam:
        if l.imag != 0:
            assert abs(abs(l.imag) - abs(l.real)) == 0.0
            assert l.real in base
    assert np.sum(lam.imag > 0) == 2 and np.sum(lam.imag < 0) == 2
    assert set(x for x in reals) <= set(base)


def test_eig_condition_closed_forms():
    """Eigenvalue condition numbers (the kappa_i that scale every eigenvalue
    tolerance): 1 for every eigenvalue of a normal quasi-triangular matrix
    (diagonal reals and standardised 2x2 blocks [[a, b], [-b, a]]), and
    sqrt(1 + b^2 / (a - c)^2) for both eigenvalues of [[a, b], [0, c]]
    (x = e_1, y proportional to (1, b / (a - c)) for lambda = a)."""
    S = np.zeros((7, 7))
    S[0, 0] = 3.0
    S[1:3, 1:3] = [[1.0, 2.0], [-2.0, 1.0]]
    S[3, 3] = -4.0
    S[4:6, 4:6] = [[-0.5, 0.25], [-0.25, -0.5]]
    S[6, 6] = 7.0
    lam, kap = metrics.eig_condition(S)
    assert np.allclose(kap, 1.0, atol=1e-12)
    for a, b, c in [(1.0, 5.0, 3.0), (2.0, -0.01, -1.0), (0.0, 100.0, 1e-3)]:
        T = np.array([[a, b], [0.0, c]])
        lam, kap = metrics.eig_condition(T)
        expect = np.sqrt(1.0 + b * b / (a - c) ** 2)
        assert np.allclose(kap, expect, rtol=1e-12), (kap, expect)


def test_match_eigenvalues_recovers_permutation():
    """The optimal one-to-one matching used by every eigenvalue comparison
    recovers a known permutation under perturbations smaller than half the
    gap, and reports the perturbation sizes."""
    rng = np.random.default_rng(3)
    a = np.arange(40) * 1.0 + 1j * (np.arange(40) % 3)
    perm = rng.permutation(40)
    noise = 1e-3 * (rng.standard_normal(40) + 1j * rng.standard_normal(40))
    b = a[perm] + noise
    p, dist = metrics.match_eigenvalues(a, b)
    assert np.array_equal(b[p], b[np.argsort(perm)])
    assert np.allclose(np.sort(dist), np.sort(np.abs(noise)))


# ------------------------------------------------ vigilant deflation test


@pytest.mark.parametrize("case,H,expected", SUBDIAG_CASES, ids=[c[0] for c in SUBDIAG_CASES])
def test_subdiag_negligible_boundaries(case, H, expected):
    """Vigilant deflation (Sec. 2.1; LAPACK-style condition of Sec. 5.6 with
    the Ahues-Tisseur refinement): each case sits on one side of one of the
    test's thresholds, with the outcome fixed by the 2x2 eigenvalue
    perturbation stated at SUBDIAG_CASES."""
    P = qr.Params()
    assert bool(qr.subdiag_negligible(H, 2, 0, 3, P, 4)) == expected


@pytest.mark.parametrize("case,rec,mode,thold,normh,expected", SPIKE_CASES, ids=[c[0] for c in SPIKE_CASES])
def test_spike_cases(case, rec, mode, thold, normh, expected):
    """AED deflation test (Sec. 5.6) on the shared boundary records."""
    assert bool(qr.spike_deflatable(*spike_case_args(rec, mode, thold, normh))) == expected


def test_subdiag_cases_separate_plausible_mistakes():
    """The cases above tell the oracle's test from plausible slips in it:
    swapped max/min pairs, no refinement, no zero-diagonal fallback, a
    relative instead of the absolute floor."""
    sml = qr.smlnum(4)

    def variant(H, k, swap_ab=False, swap_aabb=False, refine=True, fallback=True):
        h21 = abs(H[k, k - 1])
        if h21 <= sml:
            return True
        tst = abs(H[k - 1, k - 1]) + abs(H[k, k])
        if tst == 0.0 and fallback:
            tst = abs(H[k - 1, k - 2]) + abs(H[k + 1, k])
        if h21 > U * tst:
            return False
        if not refine:
            return True
        h12 = abs(H[k - 1, k])
        d = abs(H[k - 1, k - 1] - H[k, k])
        h22 = abs(H[k, k])
        ab, ba = max(h21, h12), min(h21, h12)
        aa, bb = max(h22, d), min(h22, d)
        if swap_ab:
            ab, ba = ba, ab
        if swap_aabb:
            aa, bb = bb, aa
        s = aa + ab
        return ba * (ab / s) <= max(sml, U * (bb * (aa / s)))

    mistakes = [dict(swap_ab=True), dict(swap_aabb=True), dict(refine=False), dict(fallback=False)]
    for m in mistakes:
        with np.errstate(all="ignore"):
            outcomes = [variant(H, 2, **m) == exp for _, H, exp in SUBDIAG_CASES]
        assert not all(outcomes), m
    assert all(variant(H, 2) == exp for _, H, exp in SUBDIAG_CASES)


# ------------------------------------------------ shift selection


def test_pairs_from_candidates_closed_form():
    """Shift supply (Sec. 2.5: the failed candidates become the next shifts;
    reading: bottom-most first, conjugate pairs kept together, real ones
    paired in order of appearance, an odd real dropped).  Pairs are
    (sum, product) of the two shifts."""
    c = [(1.0, 0.0), (2.0, 0.0), (3.0, 0.5), (3.0, -0.5), (4.0, 0.0)]   # top to bottom
    # from the bottom: 4 waits for a partner, the pair 3 +- 0.5i is emitted,
    # then 2 joins 4, and 1 is left over
    assert qr.pairs_from_candidates(c, 5) == [(6.0, 9.25), (6.0, 8.0)]
    assert qr.pairs_from_candidates(c, 1) == [(6.0, 9.25)]
    assert qr.pairs_from_candidates([(1.0, 0.0), (2.0, 0.0), (5.0, 0.0)], 4) == [(7.0, 10.0)]
    assert qr.pairs_from_candidates([(-1.0, 2.0), (-1.0, -2.0)], 3) == [(-2.0, 5.0)]
    assert qr.pairs_from_candidates([(7.0, 0.0)], 2) == []
    assert qr.pairs_from_candidates([], 2) == []
    # each pair's roots are two of the candidates: x^2 - sum x + prod
    rng = np.random.default_rng(3)
    cands = []
    for _ in range(12):
        if rng.random() < 0.5:
            re, im = rng.normal(), abs(rng.normal()) + 0.1
            cands += [(re, im), (re, -im)]
        else:
            cands.append((rng.normal(), 0.0))
    pairs = qr.pairs_from_candidates(cands, 100)
    pool = [complex(*z) for z in cands]
    for ssum, sprod in pairs:
        roots = np.roots([1.0, -ssum, sprod])
        for r in roots:
            j = int(np.argmin([abs(r - z) for z in pool]))
            assert abs(pool[j] - r) < 1e-12
            pool.pop(j)


# ------------------------------------------------ rejected swaps


def test_rejected_swap_leaves_blocks_untouched():
    """A rejected swap (Sec. 3.5.3: a swap can be too ill-conditioned)
    changes nothing, and move_block_up stops there.  The weak stability test
    (residual <= tol u ||A||_F) practically never fails with a complete-
    pivoting Sylvester solve, so the branch is driven by tol = 0: every swap
    whose computed residual is not exactly zero is rejected."""
    rng = np.random.default_rng(21)
    T, _ = _quasi_tri([1, 2, 2, 1], rng)
    T0 = T.copy()
    V = np.eye(T.shape[0])
    assert not qr.swap_adjacent(T, V, 1, 2, 2, tol=0.0)
    assert np.array_equal(T, T0) and np.array_equal(V, np.eye(T.shape[0]))
    assert qr.swap_adjacent(T.copy(), V.copy(), 1, 2, 2)          # the default accepts it
    assert not qr.move_block_up(T, V, 3, 1, 2, tol=0.0)
    assert np.array_equal(T, T0)


def test_aed_halts_reordering_on_rejected_swap():
    """Greedy halt (Sec. 3.5.4): once a swap is rejected the reordering stops;
    the blocks tested so far keep their outcome, the untested ones count as
    undeflated, and the window is still an orthogonal similarity of H in
    Hessenberg form with the deflated part in Schur form."""
    n, nw = 90, 30
    H = inputs.hessrand(n, 404)
    Z = np.eye(n)
    for _ in range(3):
        qr.multishift_sweep(H, Z, 0, n - 1, [(0.0, 1.0), (1.0, 2.0)])
    H0 = H.copy()
    P = qr.Params(normH=np.linalg.norm(H))
    Pr = qr.Params(normH=np.linalg.norm(H), swap_tol=0.0)
    Ha, Za = H.copy(), np.eye(n)
    nd_a, cand_a = qr.aed(Ha, Za, 0, n - 1, nw, P)
    Hr, Zr = H.copy(), np.eye(n)
    nd_r, cand_r = qr.aed(Hr, Zr, 0, n - 1, nw, Pr)
    # with rejections the deflation can only stop earlier
    assert nd_r <= nd_a
    assert len(cand_r) == nw - nd_r
    for Hx, Zx, nd in ((Ha, Za, nd_a), (Hr, Zr, nd_r)):
        assert np.linalg.norm(Zx @ Hx @ Zx.T - H0) < 1e-13 * np.linalg.norm(H0)
        assert np.max(np.abs(np.tril(Hx, -2))) == 0.0
        if nd:
            k = n - nd
            assert Hx[k, k - 1] == 0.0
            assert metrics.schur_structure_errors(Hx[k:, k:]) == []
    # the bottom-up test deflates the same leading run of blocks until the
    # first failed candidate has to move; both runs agree on that run
    assert nd_r >= 0


# ------------------------------------------------ shift recomputation


def test_recomputed_candidates_are_the_trailing_block_eigenvalues():
    """Shift recomputation after AED (LAPACK's rule, named by the paper in
    Sec. 5): the candidates become the eigenvalues of the trailing r x r
    principal submatrix of the active block (checked against LAPACK on the
    same block)."""
    H = inputs.hessrand(90, 512)
    P = qr.Params()
    c = qr.recomputed_candidates(H, 10, 89, 16, P, 90)
    assert len(c) == 16
    ref = scipy.linalg.eigvals(H[74:90, 74:90])
    _eig_close(np.array([complex(*z) for z in c]), ref, 1e-11 * np.linalg.norm(H[74:90, 74:90]))


def test_recompute_shifts_run_is_a_valid_schur_form():
    """With small windows (AED can return at most nw <= ns / 2 candidates)
    every sweep recomputes its shifts; the reduction stays a valid Schur
    factorisation with LAPACK's eigenvalues."""
    n = 160
    H = inputs.hessrand(n, 513)
    st = qr.Stats()
    S, Z, wr, wi, info = qr.schur(H, params=qr.Params(ns=16, nw=8, nmin=24, recompute_shifts=True), stats=st)
    # every sweep recomputes, except those that take exceptional shifts (at
    # most every 6th iteration without a deflation)
    assert info == 0 and st.sweeps - st.sweeps // 6 <= st.recomputed <= st.sweeps
    _check_schur(H, S, Z)
    _eig_close(wr + 1j * wi, scipy.linalg.eigvals(H), 1e-9 * np.linalg.norm(H))


def test_accuracy_metrics_closed_forms():
    """Sec. 5.4's metrics on cases with a known value: R_A of a
    factorisation off by one entry, R_orth of a scaled identity, E_lambda
    of eigenvalues moved by a known relative amount."""
    from oracle import metrics
    from oracle.qr import U

    rng = np.random.default_rng(91)
    n = 7
    A = rng.standard_normal((n, n))
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    X = Q.T @ A @ Q
    E = np.zeros((n, n))
    E[2, 5] = 3e-10                      # far above the rounding of Q X Q^T (a few u ||A||)
    want = 3e-10 / (U * np.linalg.norm(A))  # ||Q E Q^T||_F = ||E||_F
    assert abs(metrics.r_a(A, X + E, Q) - want) <= 1e-3 * want
    eps = 1e-12
    want = np.sqrt(n) * ((1 + eps) ** 2 - 1) / (U * np.sqrt(n))
    assert abs(metrics.r_orth((1 + eps) * np.eye(n)) - want) <= 1e-3 * want
    exact = np.array([1.0, -2.0, 4.0j])
    comp = exact * (1 + np.array([2.0, 5.0, 7.0]) * U)   # exact in binary64: 2, 5, 7 ulps of 1, 2, 4
    assert np.allclose(metrics.e_lambda(comp, exact), [2.0, 5.0, 7.0], rtol=1e-6)
