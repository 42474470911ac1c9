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
          fixed_thold=0.0, want_z=True, workspace=None, check=True, nmin_window=0, recompute_shifts=False,
          split_products=False):
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
                       fixed_thold=fixed_thold, want_z=1 if want_z else 0, z_init=zinit, nmin_window=nmin_window,
                       recompute_shifts=1 if recompute_shifts else 0, split_products=1 if split_products else 0)
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


def aed(H, Z, ktop, kbot, nw, deflation="lapack", fixed_thold=0.0, nmin_window=0):
    """One AED step in place; returns (nd, candidates as complex list).
    nmin_window: crossover of the window's Schur form (0 = the library's
    default, 160)."""
    lib = _lib.load()
    n = H.shape[0]
    nd = ctypes.c_int(0)
    nc = ctypes.c_int(0)
    cre = (ctypes.c_double * max(nw, 1))()
    cim = (ctypes.c_double * max(nw, 1))()
    o = _lib.make_opts(_stream_ptr().value, deflation=deflation, fixed_thold=fixed_thold, nmin_window=nmin_window)
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


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])


def _ints(xs):
    return (ctypes.c_int * len(xs))(*[int(x) for x in xs])


def schur_batched_inplace(Hs, Zs, wrs, wis, z_init=0, deflation="lapack", fixed_thold=0.0, nmin=0):
    """One persistent launch over column-major buffers (lists of tensors),
    in place; returns the per-matrix info list."""
    lib = _lib.load()
    b = len(Hs)
    info = (ctypes.c_int * max(b, 1))()
    o = _lib.make_opts(_stream_ptr().value, z_init=z_init, deflation=deflation, fixed_thold=fixed_thold, nmin=nmin)
    rc = lib.schur_hessenberg_batched(b, _ints([h.shape[0] for h in Hs]), _ptrs(Hs), _ints([_ld(h) for h in Hs]),
                                      _ptrs(Zs), _ints([_ld(z) for z in Zs]), _ptrs(wrs), _ptrs(wis), info,
                                      ctypes.byref(o))
    _check(rc, "schur_hessenberg_batched")
    return [info[i] for i in range(b)]


def schur_batched(Hs, **kw):
    """Batched reduction of a list of upper Hessenberg float64 CUDA tensors;
    returns (S list, Z list, wr list, wi list, info list); inputs untouched."""
    Ss = [colmajor(h.detach()).clone() for h in Hs]
    Zs = [new_colmajor(h.shape[0], device=h.device) for h in Hs]
    wrs = [torch.empty(h.shape[0], dtype=torch.float64, device=h.device) for h in Hs]
    wis = [torch.empty(h.shape[0], dtype=torch.float64, device=h.device) for h in Hs]
    info = schur_batched_inplace(Ss, Zs, wrs, wis, **kw)
    return Ss, Zs, wrs, wis, info


def set_batched_table(max_n, ns, nw):
    """Per-size-bucket (shifts, window) table of the batched path ([] resets)."""
    lib = _lib.load()
    _check(lib.schur_batched_set_table(len(max_n), _ints(max_n), _ints(ns), _ints(nw)), "schur_batched_set_table")


# ---------------------------------------------------------------------------
# Backward (eigenvalue adjoint) and autograd
# ---------------------------------------------------------------------------
def eig_backward(S, Z, wr, wi, gwr, gwi):
    """dL/dH = Z G Z^T for eigenvalue cotangents (gwr, gwi), S and Z from
    ``schur``; returns a column-major n x n tensor."""
    lib = _lib.load()
    n = S.shape[0]
    S = colmajor(S.detach())
    Z = colmajor(Z.detach())
    dH = new_colmajor(n, device=S.device)
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_eig_backward(n, S.data_ptr(), _ld(S), Z.data_ptr(), _ld(Z), wr.data_ptr(), wi.data_ptr(),
                                gwr.contiguous().data_ptr(), gwi.contiguous().data_ptr(), dH.data_ptr(), _ld(dH),
                                ctypes.byref(o))
    _check(rc, "schur_eig_backward")
    return dH


def eig_backward_batched(Ss, Zs, wrs, wis, gwrs, gwis):
    lib = _lib.load()
    b = len(Ss)
    Ss = [colmajor(s.detach()) for s in Ss]
    Zs = [colmajor(z.detach()) for z in Zs]
    gwrs = [g.contiguous() for g in gwrs]
    gwis = [g.contiguous() for g in gwis]
    dHs = [new_colmajor(s.shape[0], device=s.device) for s in Ss]
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_eig_backward_batched(b, _ints([s.shape[0] for s in Ss]), _ptrs(Ss), _ints([_ld(s) for s in Ss]),
                                        _ptrs(Zs), _ints([_ld(z) for z in Zs]), _ptrs(wrs), _ptrs(wis),
                                        _ptrs(gwrs), _ptrs(gwis), _ptrs(dHs), _ints([_ld(d) for d in dHs]),
                                        ctypes.byref(o))
    _check(rc, "schur_eig_backward_batched")
    return dHs


class Eigvals(torch.autograd.Function):
    """(wr, wi) = eigenvalues of the upper Hessenberg part of H; backward maps
    (dL/dwr, dL/dwi) to dL/dH through the library's adjoint.  Entries below
    the first subdiagonal do not enter the reduction, so their gradient is
    zero."""

    @staticmethod
    def forward(ctx, H):
        S, Z, wr, wi, rc = schur(H)
        if rc != 0:
            raise RuntimeError(f"schur_hessenberg returned {rc}")
        ctx.save_for_backward(S, Z, wr, wi)
        return wr.clone(), wi.clone()

    @staticmethod
    def backward(ctx, gwr, gwi):
        S, Z, wr, wi = ctx.saved_tensors
        n = S.shape[0]
        gwr = torch.zeros(n, dtype=torch.float64, device=S.device) if gwr is None else gwr
        gwi = torch.zeros(n, dtype=torch.float64, device=S.device) if gwi is None else gwi
        dH = eig_backward(S, Z, wr, wi, gwr, gwi)
        return torch.triu(dH, diagonal=-1)


def eigvals(H):
    return Eigvals.apply(H)


def hessenberg_reduce(A, want_q=True, workspace=None):
    """Householder reduction A = Q H Q^T of a general square matrix (the
    phase before the QR iteration, Sec. 1); returns (H, Q), Q None when
    want_q is False.  A itself is not modified."""
    lib = _lib.load()
    n = A.shape[0]
    H = colmajor(A.detach())
    if H.data_ptr() == A.data_ptr():
        H = H.clone()
    Q = new_colmajor(n, device=A.device) if want_q else None
    o = _lib.make_opts(_stream_ptr().value)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    rc = lib.schur_hessenberg_reduce(n, H.data_ptr(), _ld(H), Q.data_ptr() if Q is not None else None,
                                     _ld(Q) if Q is not None else 1, ctypes.byref(o))
    _check(rc, "schur_hessenberg_reduce")
    return H, Q


def eigenvectors(S, Z, wr, wi, workspace=None):
    """Right eigenvectors of H = Z S Z^T from its real Schur form (S, Z, wr,
    wi as returned by ``schur``); Z None gives those of S.  Returns X in
    LAPACK's real format (a complex pair (i, i+1) stores the real and
    imaginary parts of the eigenvector of wr[i] + i wi[i] in columns i and
    i + 1); every vector has unit 2-norm."""
    lib = _lib.load()
    n = S.shape[0]
    Sc = colmajor(S.detach())
    Zc = colmajor(Z.detach()) if Z is not None else None
    X = new_colmajor(n, device=S.device)
    o = _lib.make_opts(_stream_ptr().value)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    rc = lib.schur_eigenvectors(n, Sc.data_ptr(), _ld(Sc), Zc.data_ptr() if Zc is not None else None,
                                _ld(Zc) if Zc is not None else 1, wr.contiguous().data_ptr(),
                                wi.contiguous().data_ptr(), X.data_ptr(), _ld(X), ctypes.byref(o))
    _check(rc, "schur_eigenvectors")
    return X


def complex_eigenvectors(X, wi):
    """Complex n x n eigenvector matrix from LAPACK's real format (layout
    conversion only)."""
    n = X.shape[0]
    Xc = X.to(torch.complex128)
    w = wi.detach().cpu().tolist()
    i = 0
    while i < n:
        if w[i] > 0.0 and i + 1 < n:
            re, im = X[:, i].clone(), X[:, i + 1].clone()
            Xc[:, i] = torch.complex(re, im)
            Xc[:, i + 1] = torch.complex(re, -im)
            i += 2
        else:
            i += 1
    return Xc


def eig(A, **schur_kw):
    """Eigenvalues and right eigenvectors of a general square matrix, every
    phase on the device: Householder reduction, multishift QR with AED
    (accumulating the reduction's Q), eigenvectors from the Schur form.
    Returns (wr, wi, X, info) with X in LAPACK's real format."""
    H, Q = hessenberg_reduce(A)
    S, Z, wr, wi, info = schur(H, Q, **schur_kw)
    X = eigenvectors(S, Z, wr, wi)
    return wr, wi, X, info


def ht_reduce(A, B, Q=None, Z=None, want_qz=True):
    """Hessenberg-triangular reduction of a general pair on the GPU (the
    generalized case's first phase): returns (H, R, Q', Z') with
    (A, B) = Q' (H, R) Z'^T, H upper Hessenberg, R upper triangular.  Q, Z
    given: the transformations are multiplied into copies of them; else they
    start as the identity.  A and B are not modified."""
    lib = _lib.load()
    n = A.shape[0]
    H = colmajor(A.detach())
    if H.data_ptr() == A.data_ptr():
        H = H.clone()
    R = colmajor(B.detach())
    if R.data_ptr() == B.data_ptr():
        R = R.clone()
    zinit = 1 if (Q is not None and Z is not None) else 0
    if want_qz:
        Qc = colmajor(Q.detach().clone()) if zinit else new_colmajor(n, device=A.device)
        Zc = colmajor(Z.detach().clone()) if zinit else new_colmajor(n, device=A.device)
    else:
        Qc = Zc = None
    o = _lib.make_opts(_stream_ptr().value, want_z=1 if want_qz else 0, z_init=zinit)
    rc = lib.schur_ht_reduce(n, H.data_ptr(), _ld(H), R.data_ptr(), _ld(R),
                             Qc.data_ptr() if Qc is not None else None, _ld(Qc) if Qc is not None else 1,
                             Zc.data_ptr() if Zc is not None else None, _ld(Zc) if Zc is not None else 1,
                             ctypes.byref(o))
    _check(rc, "schur_ht_reduce")
    return H, R, Qc, Zc


def ht_reduce_batched_inplace(As, Bs, Qs, Zs, z_init=0):
    """schur_ht_reduce_batched on column-major buffers (in place); returns
    the list of per-pair statuses."""
    lib = _lib.load()
    b = len(As)
    n = (ctypes.c_int * b)(*[a.shape[0] for a in As])

    def ptrs(xs):
        return (ctypes.c_void_p * b)(*[x.data_ptr() for x in xs])

    def lds(xs):
        return (ctypes.c_int * b)(*[_ld(x) for x in xs])

    info = (ctypes.c_int * b)()
    o = _lib.make_opts(_stream_ptr().value, z_init=z_init)
    rc = lib.schur_ht_reduce_batched(b, n, ptrs(As), lds(As), ptrs(Bs), lds(Bs), ptrs(Qs), lds(Qs), ptrs(Zs),
                                     lds(Zs), info, ctypes.byref(o))
    _check(rc, "schur_ht_reduce_batched")
    return list(info)


def generalized_schur(A, B, want_qz=True):
    """Generalized real Schur form of a general pair (A, B) on the GPU:
    ht_reduce, then qz.  Returns (S, T, Q, Z, alphar, alphai, beta, info)
    with (A, B) = Q (S, T) Z^T (Q, Z None when want_qz is False)."""
    H, R, Q, Z = ht_reduce(A, B, want_qz=want_qz)
    if not want_qz:
        return qz(H, R, want_qz=False)
    return qz(H, R, Q, Z)


def qz(H, T, Q=None, Z=None, want_qz=True):
    """Generalized real Schur form of the Hessenberg-triangular pair (H, T):
    returns (S, T', Q', Z', alphar, alphai, beta, info) with
    (S, T') = Q'^T (H, T) Z'.  Q, Z given: the transformations are
    accumulated into copies of them; else they start as the identity.
    H and T are not modified."""
    lib = _lib.load()
    n = H.shape[0]
    S = colmajor(H.detach())
    if S.data_ptr() == H.data_ptr():
        S = S.clone()
    Tc = colmajor(T.detach())
    if Tc.data_ptr() == T.data_ptr():
        Tc = Tc.clone()
    zinit = 1 if (Q is not None and Z is not None) else 0
    if want_qz:
        Qc = colmajor(Q.detach().clone()) if zinit else new_colmajor(n, device=H.device)
        Zc = colmajor(Z.detach().clone()) if zinit else new_colmajor(n, device=H.device)
    else:
        Qc = Zc = None
    ar = torch.empty(n, dtype=torch.float64, device=H.device)
    ai = torch.empty_like(ar)
    be = torch.empty_like(ar)
    o = _lib.make_opts(_stream_ptr().value, want_z=1 if want_qz else 0, z_init=zinit)
    rc = lib.schur_qz(n, S.data_ptr(), _ld(S), Tc.data_ptr(), _ld(Tc), Qc.data_ptr() if Qc is not None else None,
                      _ld(Qc) if Qc is not None else 1, Zc.data_ptr() if Zc is not None else None,
                      _ld(Zc) if Zc is not None else 1, ar.data_ptr(), ai.data_ptr(), be.data_ptr(), ctypes.byref(o))
    _check(rc, "schur_qz")
    return S, Tc, Qc, Zc, ar, ai, be, rc


def qz_batched_inplace(Hs, Ts, Qs, Zs, ars, ais, bes, z_init=0):
    """schur_qz_batched on column-major buffers (in place); returns the list
    of per-pair statuses."""
    lib = _lib.load()
    b = len(Hs)
    n = (ctypes.c_int * b)(*[h.shape[0] for h in Hs])

    def ptrs(xs):
        return (ctypes.c_void_p * b)(*[x.data_ptr() for x in xs])

    def lds(xs):
        return (ctypes.c_int * b)(*[_ld(x) for x in xs])

    info = (ctypes.c_int * b)()
    o = _lib.make_opts(_stream_ptr().value, z_init=z_init)
    rc = lib.schur_qz_batched(b, n, ptrs(Hs), lds(Hs), ptrs(Ts), lds(Ts), ptrs(Qs), lds(Qs), ptrs(Zs), lds(Zs),
                              ptrs(ars), ptrs(ais), ptrs(bes), info, ctypes.byref(o))
    _check(rc, "schur_qz_batched")
    return list(info)


def qz_sweep(H, T, Q, Z, lo, hi, ssum, sprod):
    """One double-shift QZ sweep in place on column-major H, T (Q, Z both
    given or both None)."""
    lib = _lib.load()
    n = H.shape[0]
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_qz_sweep(n, H.data_ptr(), _ld(H), T.data_ptr(), _ld(T), Q.data_ptr() if Q is not None else None,
                            _ld(Q) if Q is not None else 1, Z.data_ptr() if Z is not None else None,
                            _ld(Z) if Z is not None else 1, lo, hi, float(ssum), float(sprod), ctypes.byref(o))
    _check(rc, "schur_qz_sweep")


def schur_factor_backward(S, Z, Sbar, Zbar):
    """dL/dH for a loss L(S, Z) of the standardised Schur factors of H
    (S, Z from ``schur``), cotangents Sbar = dL/dS, Zbar = dL/dZ."""
    lib = _lib.load()
    n = S.shape[0]
    Sc, Zc = colmajor(S.detach()), colmajor(Z.detach())
    Sb, Zb = colmajor(Sbar.detach().contiguous().clone()), colmajor(Zbar.detach().contiguous().clone())
    dH = new_colmajor(n, device=S.device)
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_factor_backward(n, Sc.data_ptr(), _ld(Sc), Zc.data_ptr(), _ld(Zc), Sb.data_ptr(), _ld(Sb),
                                   Zb.data_ptr(), _ld(Zb), dH.data_ptr(), _ld(dH), ctypes.byref(o))
    _check(rc, "schur_factor_backward")
    return dH


class SchurFactors(torch.autograd.Function):
    """(S, Z) = standardised real Schur factors of the upper Hessenberg part
    of H, with the Schur-factor adjoint as backward (every step in the
    library).  Entries below the first subdiagonal do not enter the
    reduction, so their gradient is zero."""

    @staticmethod
    def forward(ctx, H):
        S, Z, wr, wi, info = schur(H)
        if info != 0:
            raise RuntimeError(f"schur_hessenberg returned {info}")
        ctx.save_for_backward(S, Z)
        return S, Z

    @staticmethod
    def backward(ctx, Sbar, Zbar):
        S, Z = ctx.saved_tensors
        if Sbar is None:
            Sbar = torch.zeros_like(S)
        if Zbar is None:
            Zbar = torch.zeros_like(Z)
        return torch.triu(schur_factor_backward(S, Z, Sbar, Zbar), diagonal=-1)


def schur_factors(H):
    return SchurFactors.apply(H)


def schur_factor_backward_batched(Ss, Zs, Sbars, Zbars):
    """schur_factor_backward for lists of matrices (one launch sequence)."""
    lib = _lib.load()
    b = len(Ss)
    Ss = [colmajor(x.detach()) for x in Ss]
    Zs = [colmajor(x.detach()) for x in Zs]
    Sbs = [colmajor(x.detach().contiguous().clone()) for x in Sbars]
    Zbs = [colmajor(x.detach().contiguous().clone()) for x in Zbars]
    dHs = [new_colmajor(x.shape[0], device=x.device) for x in Ss]

    def ptrs(xs):
        return (ctypes.c_void_p * b)(*[x.data_ptr() for x in xs])

    def lds(xs):
        return (ctypes.c_int * b)(*[_ld(x) for x in xs])

    n = (ctypes.c_int * b)(*[x.shape[0] for x in Ss])
    o = _lib.make_opts(_stream_ptr().value)
    rc = lib.schur_factor_backward_batched(b, n, ptrs(Ss), lds(Ss), ptrs(Zs), lds(Zs), ptrs(Sbs), lds(Sbs),
                                           ptrs(Zbs), lds(Zbs), ptrs(dHs), lds(dHs), ctypes.byref(o))
    _check(rc, "schur_factor_backward_batched")
    return dHs
