"""Caller-provided scratch (opts->workspace) on the GPU: every entry point
that takes a workspace gives bit-identical results with one (sized by its
*_workspace query, allocated by torch) and without one (scratch allocated
inside the call); a misaligned workspace is refused with
SCHUR_ERR_WORKSPACE and changes nothing."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_03576_gb300 import _lib, api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _buf(nbytes):
    return torch.empty((nbytes + 7) // 8, dtype=torch.float64, device="cuda")


def test_schur_with_workspace_is_bit_identical():
    n = 300
    H = _dev(inputs.hessrand(n, 4242))
    S1, Z1, wr1, wi1, rc1 = api.schur(H)
    ws = _buf(api.workspace_bytes(n))
    S2, Z2, wr2, wi2, rc2 = api.schur(H, workspace=ws)
    assert rc1 == rc2 == 0
    assert torch.equal(S1, S2) and torch.equal(Z1, Z2) and torch.equal(wr1, wr2) and torch.equal(wi1, wi2)


def test_phases_with_workspace_are_bit_identical():
    lib = _lib.load()
    n = 200
    A = _dev(inputs.gaussian(n, 4243))
    b = ctypes.c_size_t()
    assert lib.schur_hessenberg_reduce_workspace(n, ctypes.byref(b)) == 0
    H1, Q1 = api.hessenberg_reduce(A)
    H2, Q2 = api.hessenberg_reduce(A, workspace=_buf(b.value))
    assert torch.equal(H1, H2) and torch.equal(Q1, Q2)
    S, Z, wr, wi, rc = api.schur(_dev(inputs.hessrand(n, 4244)))
    assert lib.schur_eigenvectors_workspace(n, 1, ctypes.byref(b)) == 0
    X1 = api.eigenvectors(S, Z, wr, wi)
    X2 = api.eigenvectors(S, Z, wr, wi, workspace=_buf(b.value))
    assert torch.equal(X1, X2)


@pytest.mark.parametrize("n", [200, 1100])
def test_eig_backward_with_workspace_is_bit_identical(n):
    """Both vector paths of the eigenvalue adjoint (per warp up to order
    1024, blocked above) through the C ABI."""
    lib = _lib.load()
    S, Z, wr, wi, rc = api.schur(_dev(inputs.hessrand(n, 4245)))
    assert rc == 0
    gr, gi = 2 * wr, 2 * wi
    dH1 = api.eig_backward(S, Z, wr, wi, gr, gi)
    b = ctypes.c_size_t()
    assert lib.schur_eig_backward_workspace(n, ctypes.byref(b)) == 0
    ws = _buf(b.value)
    dH2 = api.new_colmajor(n)
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream)
    o.workspace = ws.data_ptr()
    o.workspace_bytes = b.value
    rc = lib.schur_eig_backward(n, S.data_ptr(), n, Z.data_ptr(), n, wr.data_ptr(), wi.data_ptr(), gr.data_ptr(),
                                gi.data_ptr(), dH2.data_ptr(), n, ctypes.byref(o))
    assert rc == 0
    assert torch.equal(dH1, dH2)
    # misaligned: refused, output untouched
    dH3 = torch.zeros_like(dH1)
    o.workspace = ws.data_ptr() + 8
    o.workspace_bytes = b.value - 8
    rc = lib.schur_eig_backward(n, S.data_ptr(), n, Z.data_ptr(), n, wr.data_ptr(), wi.data_ptr(), gr.data_ptr(),
                                gi.data_ptr(), dH3.data_ptr(), n, ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_WORKSPACE
    assert torch.count_nonzero(dH3).item() == 0


def test_misaligned_workspace_leaves_h_unchanged():
    lib = _lib.load()
    n = 120
    H = _dev(inputs.hessrand(n, 4246))
    Hc = H.clone()
    Z = api.new_colmajor(n)
    wr = torch.empty(n, dtype=torch.float64, device="cuda")
    wi = torch.empty_like(wr)
    b = api.workspace_bytes(n)
    ws = _buf(b + 256)
    o = _lib.make_opts(torch.cuda.current_stream().cuda_stream)
    o.workspace = ws.data_ptr() + 64
    o.workspace_bytes = b
    rc = lib.schur_hessenberg(n, H.data_ptr(), n, Z.data_ptr(), n, wr.data_ptr(), wi.data_ptr(), ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_WORKSPACE
    assert torch.equal(H, Hc)
