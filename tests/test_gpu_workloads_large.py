"""The n = 4096 workloads (hess_n, and orthogonally similar matrices with a
prescribed spectrum, normal and non-normal; Sec. 5.3) and the largest
differentiation matrices, reduced on the GPU through the C ABI.

The CPU oracle does not finish at these orders in test time, so the
eigenvalues are checked against references that do not come from the CUDA
path: the known spectrum (prescribed family), and LAPACK's dgeev (library
cross-check) for hess_n, stored by seed under tests/golden by
make_lapack_reference.py together with LAPACK's eigenvalue condition
numbers.  Tolerances as in the parity tests: backward error and
orthogonality / sqrt(n) <= 1e-13 (Sec. 5.4), a standardised quasi-triangular
S, and |lambda_gpu - lambda_ref| <= 1e-10 kappa_i ||H||_F under a one-to-one
matching."""

import math
import os

import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")

from oracle import adjoint, metrics, testmats  # noqa: E402
from paper_2007_03576_gb300 import api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _checks_on_device(H, S, Z):
    """Backward error and orthogonality with device GEMMs (library products,
    used only to check); the structure of S on the host."""
    Hd = _dev(H)
    n = H.shape[0]
    ra = float(torch.linalg.matrix_norm(Z @ S @ Z.t() - Hd) / torch.linalg.matrix_norm(Hd))
    ro = float(torch.linalg.matrix_norm(Z.t() @ Z - torch.eye(n, dtype=torch.float64, device="cuda"))) / math.sqrt(n)
    assert ra <= 1e-13, ra
    assert ro <= 1e-13, ro
    Sn = S.cpu().numpy()
    assert metrics.schur_structure_errors(Sn) == []
    return ra, ro, Sn


def _match(lam, ref, kappa, nh):
    perm, dist = metrics.match_eigenvalues(np.asarray(ref), np.asarray(lam))
    bound = 1e-10 * np.asarray(kappa) * nh
    assert np.all(dist <= bound), float(np.max(dist / (np.asarray(kappa) * nh)))
    return float(np.max(dist / (np.asarray(kappa) * nh)))


def test_hess_n4096_vs_lapack():
    n, seed = 4096, 2021
    ref = np.load(os.path.join(GOLDEN, f"lapack_hessrand_n{n}_seed{seed}.npz"))
    H = inputs.hessrand(n, seed)
    S, Z, wr, wi, info = api.schur(_dev(H), n_shifts=64, aed_window=128)
    assert info == 0
    _checks_on_device(H, S, Z)
    lam = wr.cpu().numpy() + 1j * wi.cpu().numpy()
    _match(lam, ref["eig"], ref["kappa"], np.linalg.norm(H))
    assert abs(np.sum(lam) - np.trace(H)) <= 1e-12 * n * np.linalg.norm(H)


def _prescribed(nonnormal, seed=2022, n=4096):
    # A = Q T Q^T reduced to Hessenberg form by LAPACK's dgehrd (input
    # generation only; any orthogonal reduction keeps the spectrum)
    return testmats.prescribed(n, np.random.default_rng(seed), nonnormal=nonnormal,
                               reduce=lambda A: scipy.linalg.hessenberg(A, check_finite=False))


def test_prescribed_normal_n4096_known_spectrum():
    """Normal family: every eigenvalue has condition number 1, so the
    computed spectrum is within 1e-10 ||H||_F of the prescribed one."""
    H, lam_ref = _prescribed(False)
    S, Z, wr, wi, info = api.schur(_dev(H), n_shifts=64, aed_window=128)
    assert info == 0
    _checks_on_device(H, S, Z)
    lam = wr.cpu().numpy() + 1j * wi.cpu().numpy()
    _match(lam, lam_ref, np.ones(len(lam_ref)), np.linalg.norm(H))


def test_prescribed_nonnormal_n4096_known_spectrum():
    """Non-normal family (strictly upper U[-1, 1] part): the prescribed
    eigenvalues with the condition numbers of T = D + N from LAPACK's left
    and right eigenvectors (stored by seed)."""
    n, seed = 4096, 2022
    ref = np.load(os.path.join(GOLDEN, f"lapack_prescribed_nonnormal_n{n}_seed{seed}.npz"))
    H, lam_ref = _prescribed(True, seed, n)
    # condition number of each prescribed eigenvalue: that of LAPACK's
    # nearest eigenvalue of T
    perm, _ = metrics.match_eigenvalues(lam_ref, ref["eig"])
    kappa = ref["kappa"][perm]
    S, Z, wr, wi, info = api.schur(_dev(H), n_shifts=64, aed_window=128)
    assert info == 0
    _checks_on_device(H, S, Z)
    lam = wr.cpu().numpy() + 1j * wi.cpu().numpy()
    _match(lam, lam_ref, kappa, np.linalg.norm(H))


def test_backward_n1024_matches_oracle_adjoint():
    """The largest differentiation matrices (n = 1024): the GPU adjoint
    against the oracle's adjoint evaluated on the same Schur factor."""
    n = 1024
    H = inputs.hessrand(n, 600 + n)
    S, Z, wr, wi, info = api.schur(_dev(H))
    assert info == 0
    gr, gi = 2 * wr, 2 * wi
    dH = api.eig_backward(S, Z, wr, wi, gr, gi).cpu().numpy()
    Sn, Zn = S.cpu().numpy(), Z.cpu().numpy()
    ref = adjoint.eig_adjoint(Sn, Zn, gr.cpu().numpy(), gi.cpu().numpy())
    _, kap = metrics.eig_condition(Sn)
    scale = np.max(kap) * np.linalg.norm(np.concatenate([gr.cpu().numpy(), gi.cpu().numpy()]))
    assert np.max(np.abs(dH - ref)) <= 1e-10 * scale, np.max(np.abs(dH - ref)) / scale


def test_backward_n4096_closed_forms():
    """The blocked eigenvalue adjoint at n = 4096 on the normal prescribed
    family (every eigenvalue has condition number 1): cotangents g = 1 give
    dH = I (sum of the eigenvalues = tr H) and g = 2 conj(lambda) give
    dH = 2 H^T (sum of Re lambda^2 = tr H^2), both exactly, so the computed
    adjoint is within a small multiple of u n ||H|| of them."""
    H, _ = _prescribed(False, seed=2024)
    n = H.shape[0]
    S, Z, wr, wi, info = api.schur(_dev(H), n_shifts=64, aed_window=128)
    assert info == 0
    one = torch.ones(n, dtype=torch.float64, device="cuda")
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    dH = api.eig_backward(S, Z, wr, wi, one, zero)
    err_i = torch.max(torch.abs(dH - torch.eye(n, dtype=torch.float64, device="cuda"))).item()
    assert err_i <= 1e-10, err_i
    dH = api.eig_backward(S, Z, wr, wi, 2 * wr, -2 * wi)
    nh = float(np.linalg.norm(H))
    err_h = torch.max(torch.abs(dH - 2 * _dev(H).t())).item()
    assert err_h <= 1e-10 * nh, err_h / nh
