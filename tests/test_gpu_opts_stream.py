"""Options read through the C ABI: a zero struct_size means "the whole
struct" in every entry point, so the stream given in such an opts block is
the one the work runs on.

The check: the input is written by a copy that runs on a non-default stream
behind a long sleep; the call is made on that stream without synchronising
first.  Only a call that runs on that stream sees the right input (the
library's own streams are non-blocking, so the legacy default stream would
not wait for the sleep)."""

import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_03576_gb300 import _lib, api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _opts_struct_size_zero(stream):
    o = _lib.make_opts(stream.cuda_stream)
    o.struct_size = 0
    return o


def test_schur_hessenberg_runs_on_the_stream_of_a_struct_size_zero_opts():
    n = 120
    H = inputs.hessrand(n, 31)
    src = _dev(H)
    S = _dev(inputs.hessrand(n, 32))          # wrong input until the delayed copy lands
    Z = api.new_colmajor(n)
    wr = torch.empty(n, dtype=torch.float64, device="cuda")
    wi = torch.empty_like(wr)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(200_000_000)      # ~0.1 s at 2 GHz
        S.copy_(src)
    o = _opts_struct_size_zero(s)
    rc = _lib.load().schur_hessenberg(n, S.data_ptr(), n, Z.data_ptr(), n, wr.data_ptr(), wi.data_ptr(),
                                      ctypes.byref(o))
    assert rc == 0, _lib.status(rc)
    s.synchronize()
    Sn, Zn = S.cpu().numpy(), Z.cpu().numpy()
    ra = np.linalg.norm(Zn @ Sn @ Zn.T - H) / np.linalg.norm(H)
    assert ra <= 1e-13, ra
    assert np.linalg.norm(Zn.T @ Zn - np.eye(n)) / math.sqrt(n) <= 1e-13


def test_batched_runs_on_the_stream_of_a_struct_size_zero_opts():
    sizes = [40, 77]
    Hs = [inputs.hessrand(m, [33, b]) for b, m in enumerate(sizes)]
    srcs = [_dev(H) for H in Hs]
    Ss = [_dev(inputs.hessrand(m, [34, b])) for b, m in enumerate(sizes)]
    Zs = [api.new_colmajor(m) for m in sizes]
    wr = [torch.empty(m, dtype=torch.float64, device="cuda") for m in sizes]
    wi = [torch.empty_like(w) for w in wr]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(200_000_000)
        for S, src in zip(Ss, srcs):
            S.copy_(src)
    o = _opts_struct_size_zero(s)
    B = len(sizes)
    arr = lambda T, xs: (T * B)(*xs)  # noqa: E731
    info = (ctypes.c_int * B)()
    rc = _lib.load().schur_hessenberg_batched(
        B, arr(ctypes.c_int, sizes), arr(ctypes.c_void_p, [S.data_ptr() for S in Ss]), arr(ctypes.c_int, sizes),
        arr(ctypes.c_void_p, [Z.data_ptr() for Z in Zs]), arr(ctypes.c_int, sizes),
        arr(ctypes.c_void_p, [w.data_ptr() for w in wr]), arr(ctypes.c_void_p, [w.data_ptr() for w in wi]), info,
        ctypes.byref(o))
    assert rc == 0, _lib.status(rc)
    s.synchronize()
    for b, H in enumerate(Hs):
        assert info[b] == 0
        Sn, Zn = Ss[b].cpu().numpy(), Zs[b].cpu().numpy()
        assert np.linalg.norm(Zn @ Sn @ Zn.T - H) / np.linalg.norm(H) <= 1e-13
