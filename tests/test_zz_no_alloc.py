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


def _noalloc(H):
    """One call of the new entry point on fresh buffers; returns
    (status, S, Z, wr, wi) as numpy arrays."""
    lib = _lib.load()
    n = H.shape[0]
    Hd = _dev(H).clone()
    Zd = api.new_colmajor(n)
    wr = torch.empty(n, dtype=torch.float64, device="cuda")
    wi = torch.empty(n, dtype=torch.float64, device="cuda")
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream)
    rc = lib.schur_hessenberg_noalloc(n, Hd.data_ptr(), Hd.stride(1), Zd.data_ptr(), Zd.stride(1), wr.data_ptr(),
                                      wi.data_ptr(), ctypes.byref(o))
    return rc, Hd.cpu().numpy(), Zd.cpu().numpy(), wr.cpu().numpy(), wi.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_schur_hessenberg_two_calls():
    for call, (n, seed) in enumerate([(200, 11), (333, 12)]):
        H = inputs.hessrand(n, seed)
        rc, S, Z, wr, wi = _noalloc(H)
        assert rc == 0, (call, rc)
        nh = np.linalg.norm(H)
        assert np.linalg.norm(Z @ S @ Z.T - H) / nh <= 1e-13
        assert np.linalg.norm(Z.T @ Z - np.eye(n)) / math.sqrt(n) <= 1e-13
        assert metrics.schur_structure_errors(S) == []
        S1, Z1, wr1, wi1, rc1 = api.schur(_dev(H))
        assert rc1 == 0
        S1 = S1.cpu().numpy()
        _, kap = metrics.eig_condition(S1)
        perm, dist = metrics.match_eigenvalues(wr1.cpu().numpy() + 1j * wi1.cpu().numpy(), wr + 1j * wi)
        assert np.all(dist <= 1e-10 * kap * nh), (call, float(np.max(dist / (kap * nh))))


@pytest.mark.gpu
def test_noalloc_rejects_orders_above_its_limit():
    lib = _lib.load()
    o = _lib.make_opts(0)
    rc = lib.schur_hessenberg_noalloc(1025, 1, 1025, 1, 1025, 1, 1, ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_TOO_LARGE
    assert "no-allocation" in _lib.status(rc)
