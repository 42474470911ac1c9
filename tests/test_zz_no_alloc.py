"""schur_hessenberg_noalloc: the entry point for callers that cannot allocate
memory during the call (its scratch is a fixed device array).  Called through
the C ABI twice in a row and checked against schur_hessenberg on the same
inputs, with the tolerances of the parity tests: backward error and
orthogonality <= 1e-13, standardised structure, eigenvalues within
1e-10 * kappa_i * ||H||_F.  This file is collected last on purpose."""

import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import metrics  # noqa: E402
from paper_2007_03576_gb300 import _lib, api, inputs  # noqa: E402


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _padded(A, ld):
    """Column-major device copy of A inside an ld x n buffer (ld >= n); the
    padding rows hold a sentinel that the call must leave alone."""
    n = A.shape[0]
    buf = torch.full((n, ld), 7.25, dtype=torch.float64, device="cuda")   # storage: column j at j*ld
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda()
    return buf


def _noalloc(H, ld=None, Z0=None):
    """One call of the new entry point on fresh buffers (leading dimension ld,
    default n; Z0 given: z_init = 1 with Z = Z0 on entry); returns
    (status, S, Z, wr, wi) as numpy arrays and checks that the padding rows
    were not written."""
    lib = _lib.load()
    n = H.shape[0]
    ld = n if ld is None else ld
    Hb = _padded(H, ld)
    Zb = _padded(np.eye(n) if Z0 is None else Z0, ld)
    wr = torch.empty(n, dtype=torch.float64, device="cuda")
    wi = torch.empty(n, dtype=torch.float64, device="cuda")
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream, z_init=0 if Z0 is None else 1)
    rc = lib.schur_hessenberg_noalloc(n, Hb.data_ptr(), ld, Zb.data_ptr(), ld, wr.data_ptr(), wi.data_ptr(),
                                      ctypes.byref(o))
    torch.cuda.synchronize()
    if ld > n:
        assert bool(torch.all(Hb[:, n:] == 7.25)) and bool(torch.all(Zb[:, n:] == 7.25))
    S = Hb[:, :n].cpu().numpy().T
    Z = Zb[:, :n].cpu().numpy().T
    return rc, S, Z, wr.cpu().numpy(), wi.cpu().numpy()


def _check_against_schur_hessenberg(H, S, Z, wr, wi, Z0=None, tag=""):
    n = H.shape[0]
    nh = np.linalg.norm(H)
    Q = np.eye(n) if Z0 is None else Z0
    # H = Z S Z^T with Z = Q Z_QR, i.e. Q H Q^T = Z S Z^T
    assert np.linalg.norm(Z @ S @ Z.T - Q @ H @ Q.T) / nh <= 1e-13, tag
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) / math.sqrt(n) <= 1e-13, tag
    assert metrics.schur_structure_errors(S) == [], tag
    S1, Z1, wr1, wi1, rc1 = api.schur(_dev(H))
    assert rc1 == 0
    S1 = S1.cpu().numpy()
    _, kap = metrics.eig_condition(S1)
    perm, dist = metrics.match_eigenvalues(wr1.cpu().numpy() + 1j * wi1.cpu().numpy(), wr + 1j * wi)
    assert np.all(dist <= 1e-10 * kap * nh), (tag, float(np.max(dist / (kap * nh))))


@pytest.mark.gpu
def test_noalloc_matches_schur_hessenberg_two_calls():
    for call, (n, seed) in enumerate([(200, 11), (333, 12)]):
        H = inputs.hessrand(n, seed)
        rc, S, Z, wr, wi = _noalloc(H)
        assert rc == 0, (call, rc)
        _check_against_schur_hessenberg(H, S, Z, wr, wi, tag=f"call {call}")


@pytest.mark.gpu
def test_noalloc_allocates_no_device_memory():
    """After a first call (which sets the entry point up on this device), a
    call leaves the device's free memory unchanged."""
    H = inputs.hessrand(150, 21)
    H0d = _dev(H)
    Hd = H0d.clone()
    Zd = api.new_colmajor(150)
    wr = torch.empty(150, dtype=torch.float64, device="cuda")
    wi = torch.empty(150, dtype=torch.float64, device="cuda")
    lib = _lib.load()
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream)

    def call():
        Hd.copy_(H0d)
        torch.cuda.synchronize()
        return lib.schur_hessenberg_noalloc(150, Hd.data_ptr(), 150, Zd.data_ptr(), 150, wr.data_ptr(),
                                            wi.data_ptr(), ctypes.byref(o))

    assert call() == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


@pytest.mark.gpu
def test_noalloc_padded_leading_dimensions():
    n = 181
    H = inputs.hessrand(n, 22)
    rc, S, Z, wr, wi = _noalloc(H, ld=n + 7)
    assert rc == 0
    _check_against_schur_hessenberg(H, S, Z, wr, wi, tag="ld = n + 7")


@pytest.mark.gpu
def test_noalloc_accumulates_into_given_z():
    n = 140
    H = inputs.hessrand(n, 23)
    Q, R = np.linalg.qr(np.random.default_rng(24).standard_normal((n, n)))
    Q = Q * np.sign(np.diag(R))
    rc, S, Z, wr, wi = _noalloc(H, Z0=Q)
    assert rc == 0
    _check_against_schur_hessenberg(H, S, Z, wr, wi, Z0=Q, tag="z_init = 1")


@pytest.mark.gpu
def test_noalloc_rejects_orders_above_its_limit():
    lib = _lib.load()
    o = _lib.make_opts(0)
    rc = lib.schur_hessenberg_noalloc(1025, 1, 1025, 1, 1025, 1, 1, ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_TOO_LARGE
    assert "no-allocation" in _lib.status(rc)
