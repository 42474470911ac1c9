"""PyTorch-facing API over the C ABI (device memory and streams only; every
arithmetic step runs in the library's CUDA kernels).

Matrices are torch float64 CUDA tensors with the mathematical layout
M[i, j].  The C ABI is column-major: a tensor whose strides are (1, ld) is
passed without a copy; any other layout is copied into a column-major buffer
first (and the result returned in that buffer).
"""

import ctypes

import torch

from . import _lib


def _stream_ptr():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def colmajor(T):
    """Column-major (strides (1, ld)) float64 CUDA view of T, copying if
    needed."""
    if T.dtype != torch.float64:
        raise TypeError("float64 required")
    if not T.is_cuda:
        raise ValueError("CUDA tensor required")
    n0, n1 = T.shape
    if T.stride(0) == 1 and T.stride(1) >= max(1, n0):
        return T
    return T.t().contiguous().t()


def _ld(C):
    return max(1, C.stride(1))


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"{what} failed: {rc} ({_lib.status(rc)})")
    return rc


def new_colmajor(n, m=None, device="cuda"):
    m = n if m is None else m
    return torch.empty((m, n), dtype=torch.float64, device=device).t()


def schur(H, Z=None, *, n_shifts=0, aed_window=0, bulges_per_chain=0, nmin=0, nibble=0, deflation="lapack",
          fixed_thold=0.0, want_z=True, workspace=None, check=True):
    """Real Schur form of the upper Hessenberg H: returns (S, Z, wr, wi, info)
    with S = Z^T H Z (H itself is not modified).  If Z is given the
    transformations are accumulated into a copy of it (Z <- Z Z_QR); else Z
    starts as the identity."""
    lib = _lib.load()
    n = H.shape[0]
    S = colmajor(H.detach())
    if S.data_ptr() == H.data_ptr():
        S = S.clone()  # preserve_format keeps the column-major strides
    zinit = 1 if Z is not None else 0
    if want_z:
        Zc = colmajor(Z.detach().clone()) if Z is not None else new_colmajor(n, device=H.device)
    else:
        Zc = None
    wr = torch.empty(n, dtype=torch.float64, device=H.device)
    wi = torch.empty(n, dtype=torch.float64, device=H.device)
    o = _lib.make_opts(_stream_ptr().value, n_shifts=n_shifts, aed_window=aed_window,
                       bulges_per_chain=bulges_per_chain, nmin=nmin, nibble=nibble, deflation=deflation,
                       fixed_thold=fixed_thold, want_z=1 if want_z else 0, z_init=zinit)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    rc = lib.schur_hessenberg(n, S.data_ptr(), _ld(S), Zc.data_ptr() if Zc is not None else None,
                              _ld(Zc) if Zc is not None else 1, wr.data_ptr(), wi.data_ptr(), ctypes.byref(o))
    if check:
        _check(rc, "schur_hessenberg")
    return S, Zc, wr, wi, rc


def schur_inplace(Hc, Zc, wr, wi, opts):
    """Low-level call on column-major buffers (no copies): Hc, Zc from
    ``colmajor``/``new_colmajor``; returns the status code."""
    lib = _lib.load()
    n = Hc.shape[0]
    return lib.schur_hessenberg(n, Hc.data_ptr(), _ld(Hc), Zc.data_ptr() if Zc is not None else None,
                                _ld(Zc) if Zc is not None else 1, wr.data_ptr(), wi.data_ptr(), ctypes.byref(opts))


def last_stats():
    s = _lib.SchurStats()
    _lib.load().schur_last_stats(ctypes.byref(s))
    return {f: getattr(s, f) for f, _ in s._fields_}


def workspace_bytes(n, **kw):
    o = _lib.make_opts(0, **kw)
    b = ctypes.c_size_t(0)
    _check(_lib.load().schur_workspace_size(n, ctypes.byref(o), ctypes.byref(b)), "schur_workspace_size")
    return b.value


def sweep(H, Z, ilo, ihi, pairs, bulges_per_chain=0):
    """One windowed multishift sweep in place on column-major H, Z."""
    lib = _lib.load()
    n = H.shape[0]
    flat = [float(x) for p in pairs for x in p]
    arr = (ctypes.c_double * len(flat))(*flat)
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_sweep(n, H.data_ptr(), _ld(H), Z.data_ptr() if Z is not None else None,
                         _ld(Z) if Z is not None else 1, ilo, ihi, arr, len(pairs), bulges_per_chain,
                         ctypes.byref(o))
    _check(rc, "schur_sweep")


def aed(H, Z, ktop, kbot, nw, deflation="lapack", fixed_thold=0.0):
    """One AED step in place; returns (nd, candidates as complex list)."""
    lib = _lib.load()
    n = H.shape[0]
    nd = ctypes.c_int(0)
    nc = ctypes.c_int(0)
    cre = (ctypes.c_double * max(nw, 1))()
    cim = (ctypes.c_double * max(nw, 1))()
    o = _lib.make_opts(_stream_ptr().value, deflation=deflation, fixed_thold=fixed_thold)
    rc = lib.schur_aed(n, H.data_ptr(), _ld(H), Z.data_ptr() if Z is not None else None,
                       _ld(Z) if Z is not None else 1, ktop, kbot, nw, ctypes.byref(nd), cre, cim,
                       ctypes.byref(nc), ctypes.byref(o))
    _check(rc, "schur_aed")
    return nd.value, [complex(cre[i], cim[i]) for i in range(nc.value)]


def small_qr(H, Z, ilo, ihi):
    lib = _lib.load()
    n = H.shape[0]
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_small_qr(n, H.data_ptr(), _ld(H), Z.data_ptr() if Z is not None else None,
                            _ld(Z) if Z is not None else 1, ilo, ihi, ctypes.byref(o))
    return _check(rc, "schur_small_qr")


def apply_u(side, A, r0, c0, m, U):
    lib = _lib.load()
    k = U.shape[0]
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_apply_u(side, A.data_ptr(), _ld(A), r0, c0, m, k, U.data_ptr(), _ld(U), ctypes.byref(o))
    _check(rc, "schur_apply_u")
