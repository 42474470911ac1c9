"""Argument checks of every C-ABI entry point, on the host (no GPU).

The header's convention: a bad argument i (1-based) returns -i, before any
device work.  Each case starts from valid arguments and breaks one at a
time.  Device pointers are dummies that a rejected call never touches; no
call here has all of its arguments valid, so none reaches the device."""

import ctypes

import pytest

from paper_2007_03576_gb300 import _lib

DEV = ctypes.c_void_p(4096)  # stands for a device pointer; never dereferenced
N = 8


def _opts():
    return ctypes.byref(_lib.make_opts(0))


def _expect(fn, args, i, bad):
    a = list(args)
    a[i] = bad
    rc = fn(*a)
    assert rc == -(i + 1), (fn.__name__, i + 1, bad, rc)


SCALAR_CASES = [
    # name, valid arguments (opts appended), {0-based index: [bad values]}
    ("schur_hessenberg", [N, DEV, N, DEV, N, DEV, DEV],
     {0: [-1], 1: [None], 2: [N - 1, 0], 3: [None], 4: [N - 1], 5: [None], 6: [None]}),
    ("schur_hessenberg_noalloc", [N, DEV, N, DEV, N, DEV, DEV],
     {0: [-1], 1: [None], 2: [N - 1], 3: [None], 4: [N - 1], 5: [None], 6: [None]}),
    ("schur_eig_backward", [N, DEV, N, DEV, N, DEV, DEV, DEV, DEV, DEV, N],
     {0: [-1], 1: [None], 2: [N - 1], 3: [None], 4: [N - 1], 5: [None], 6: [None], 7: [None],
      8: [None], 9: [None], 10: [N - 1]}),
    ("schur_sweep", [N, DEV, N, DEV, N, 0, N - 1, (ctypes.c_double * 4)(), 2, 0],
     {0: [0], 1: [None], 2: [N - 1], 4: [N - 1], 5: [-1, N], 6: [1, N], 7: [None], 8: [0, 32 * 32 + 1]}),
    ("schur_aed", [N, DEV, N, DEV, N, 0, N - 1, 4, ctypes.byref(ctypes.c_int()), None, None, None],
     {0: [0], 1: [None], 2: [N - 1], 4: [N - 1], 5: [-1, N], 6: [-1, N], 7: [0, N + 1], 8: [None]}),
    ("schur_small_qr", [N, DEV, N, DEV, N, 0, N - 1],
     {0: [0], 1: [None], 2: [N - 1], 4: [N - 1], 5: [-1, N], 6: [-1, N]}),
    ("schur_apply_u", [0, DEV, N, 0, 0, N, 4, DEV, 4],
     {0: [2, -1], 1: [None], 2: [0], 3: [-1], 4: [-1], 5: [-1], 6: [0, 1025], 7: [None], 8: [3]}),
    ("schur_fastmath_eval", [N, DEV, DEV],
     {0: [-1], 1: [None], 2: [None]}),
    ("schur_fp64_fma_probe", [100, 4, DEV, ctypes.byref(ctypes.c_double())],
     {0: [0], 1: [0], 2: [None], 3: [None]}),
    ("schur_chase_schedule", [0, 100, 8, 4, 4, (ctypes.c_int * 28)(), ctypes.byref(ctypes.c_int()), None, None],
     {0: [-1], 1: [1, -5], 2: [0, 1025], 3: [-1], 4: [-1], 5: [None], 6: [None]}),
    ("schur_vigilant_eval", [N, DEV, 0, 0.0, 1.0, 4, DEV],
     {0: [-1], 1: [None], 2: [-1, 3], 5: [0], 6: [None]}),
    ("schur_spike_eval", [N, DEV, 0, 0.0, 1.0, 4, DEV],
     {0: [-1], 1: [None], 2: [-1, 3], 5: [0], 6: [None]}),
    ("schur_hessenberg_reduce", [N, DEV, N, DEV, N],
     {0: [-1], 1: [None], 2: [N - 1, 0], 4: [N - 1]}),
    ("schur_eigenvectors", [N, DEV, N, DEV, N, DEV, DEV, DEV, N],
     {0: [-1], 1: [None], 2: [N - 1], 4: [N - 1], 5: [None], 6: [None], 7: [None], 8: [N - 1]}),
    ("schur_factor_backward", [N, DEV, N, DEV, N, DEV, N, DEV, N, DEV, N],
     {0: [-1, 1025], 1: [None], 2: [N - 1], 3: [None], 4: [N - 1], 5: [None], 6: [N - 1], 7: [None], 8: [N - 1],
      9: [None], 10: [N - 1]}),
    ("schur_qz", [N, DEV, N, DEV, N, DEV, N, DEV, N, DEV, DEV, DEV],
     {0: [-1], 1: [None], 2: [N - 1], 3: [None], 4: [N - 1], 5: [None], 6: [N - 1], 7: [None], 8: [N - 1],
      9: [None], 10: [None], 11: [None]}),
    ("schur_ht_reduce", [N, DEV, N, DEV, N, DEV, N, DEV, N],
     {0: [-1], 1: [None], 2: [N - 1, 0], 3: [None], 4: [N - 1], 5: [None], 6: [N - 1], 7: [None], 8: [N - 1]}),
    ("schur_qz_sweep", [N, DEV, N, DEV, N, DEV, N, DEV, N, 0, N - 1, 1.0, 2.0],
     {0: [2], 1: [None], 2: [N - 1], 3: [None], 4: [N - 1], 6: [N - 1], 8: [N - 1], 9: [-1, N - 2],
      10: [1, N]}),
]


@pytest.mark.parametrize("name,args,bad", SCALAR_CASES, ids=[c[0] for c in SCALAR_CASES])
def test_scalar_entry_points_reject_each_bad_argument(name, args, bad):
    lib = _lib.load()
    fn = getattr(lib, name)
    full = list(args) + ([_opts()] if len(fn.argtypes) > len(args) else [])
    for i, values in bad.items():
        for v in values:
            _expect(fn, full, i, v)


def _host_arrays(batch, n):
    ints = lambda v: (ctypes.c_int * batch)(*([v] * batch))
    ptrs = lambda: (ctypes.c_void_p * batch)(*([4096] * batch))
    return ints, ptrs


def test_batched_rejects_each_bad_argument():
    lib = _lib.load()
    B = 3
    ints, ptrs = _host_arrays(B, N)
    info = (ctypes.c_int * B)()
    valid = [B, ints(N), ptrs(), ints(N), ptrs(), ints(N), ptrs(), ptrs(), info, _opts()]
    fn = lib.schur_hessenberg_batched
    assert fn(0, None, None, None, None, None, None, None, None, _opts()) == 0
    _expect(fn, valid, 0, -1)
    for i in range(1, 9):  # a missing array
        _expect(fn, valid, i, None)
    # one bad entry in the middle of an array
    bad_n = ints(N); bad_n[1] = 0
    _expect(fn, valid, 1, bad_n)
    bad_n = ints(N); bad_n[1] = 1025
    _expect(fn, valid, 1, bad_n)
    for i in (2, 4, 6, 7):  # a null device pointer for one matrix
        p = ptrs(); p[2] = None
        _expect(fn, valid, i, p)
    for i in (3, 5):  # a leading dimension below n for one matrix
        ld = ints(N); ld[1] = N - 1
        _expect(fn, valid, i, ld)


def test_batched_backward_rejects_each_bad_argument():
    lib = _lib.load()
    B = 3
    ints, ptrs = _host_arrays(B, N)
    valid = [B, ints(N), ptrs(), ints(N), ptrs(), ints(N), ptrs(), ptrs(), ptrs(), ptrs(), ptrs(), ints(N),
             _opts()]
    fn = lib.schur_eig_backward_batched
    assert fn(0, *([None] * 11), _opts()) == 0
    _expect(fn, valid, 0, -1)
    for i in range(1, 12):
        _expect(fn, valid, i, None)
    bad_n = ints(N); bad_n[2] = 1025
    _expect(fn, valid, 1, bad_n)
    for i in (2, 4, 6, 7, 8, 9, 10):
        p = ptrs(); p[1] = None
        _expect(fn, valid, i, p)
    for i in (3, 5, 11):
        ld = ints(N); ld[0] = N - 1
        _expect(fn, valid, i, ld)


def test_set_table_rejects_bad_tables():
    lib = _lib.load()
    arr = lambda *v: (ctypes.c_int * len(v))(*v)
    fn = lib.schur_batched_set_table
    assert fn(9, arr(1), arr(8), arr(24)) == -1
    assert fn(-1, arr(1), arr(8), arr(24)) == -1
    assert fn(1, None, arr(8), arr(24)) == -2
    assert fn(1, arr(100), None, arr(24)) == -3
    assert fn(1, arr(100), arr(8), None) == -4
    assert fn(1, arr(100), arr(8), arr(3)) == -4      # window below 4
    assert fn(1, arr(100), arr(1), arr(24)) == -3     # fewer than 2 shifts
    assert fn(0, None, None, None) == 0               # built-in table again


def test_noalloc_order_limit_and_workspace_args():
    lib = _lib.load()
    fn = lib.schur_hessenberg_noalloc
    assert fn(1025, DEV, 1025, DEV, 1025, DEV, DEV, _opts()) == _lib.SCHUR_ERR_TOO_LARGE
    assert fn(0, None, 1, None, 1, None, None, _opts()) == 0
    b = ctypes.c_size_t(0)
    assert lib.schur_workspace_size(N, _opts(), None) == -3
    assert lib.schur_workspace_size(N, None, ctypes.byref(b)) == 0 and b.value > 0
    assert lib.schur_default_opts(None) == -1
    assert lib.schur_last_stats(None) == -1


def test_phase_workspace_sizes():
    """Scratch sizes of the reduction and eigenvector entry points (host
    arithmetic only): the eigenvector scratch holds an n x n buffer when Z is
    given; bad arguments return their index."""
    lib = _lib.load()
    b = ctypes.c_size_t(0)
    assert lib.schur_hessenberg_reduce_workspace(1000, ctypes.byref(b)) == 0
    assert 2 * 1000 * 8 <= b.value < 64 * 1024
    assert lib.schur_hessenberg_reduce_workspace(-1, ctypes.byref(b)) == -1
    assert lib.schur_hessenberg_reduce_workspace(10, None) == -2
    assert lib.schur_eigenvectors_workspace(1000, 1, ctypes.byref(b)) == 0
    with_z = b.value
    assert with_z >= 1000 * 1000 * 8
    assert lib.schur_eigenvectors_workspace(1000, 0, ctypes.byref(b)) == 0
    assert b.value < with_z - 1000 * 1000 * 8 + 4096
    assert lib.schur_eigenvectors_workspace(-1, 0, ctypes.byref(b)) == -1
    assert lib.schur_eigenvectors_workspace(10, 0, None) == -3


def test_eig_backward_workspace_and_large_orders():
    """The eigenvalue adjoint's scratch: five n x n buffers on the per-warp
    path (orders up to 1024), three on the blocked path (above, any order);
    a caller workspace below that size is refused before any device work, at
    an order the per-warp path could not take."""
    lib = _lib.load()
    b = ctypes.c_size_t(0)
    for n in (1, 511, 1024):
        assert lib.schur_eig_backward_workspace(n, ctypes.byref(b)) == 0
        assert 5 * n * n * 8 <= b.value < 5 * n * n * 8 + 64 * 1024
    for n in (1025, 1500, 20000):
        assert lib.schur_eig_backward_workspace(n, ctypes.byref(b)) == 0
        assert 3 * n * n * 8 <= b.value < 3 * n * n * 8 + 8 * 1024 * 1024, (n, b.value)
    assert lib.schur_eig_backward_workspace(-1, ctypes.byref(b)) == -1
    assert lib.schur_eig_backward_workspace(10, None) == -2
    n = 3000
    assert lib.schur_eig_backward_workspace(n, ctypes.byref(b)) == 0
    o = _lib.make_opts(0)
    o.workspace = DEV
    o.workspace_bytes = b.value - 1
    rc = lib.schur_eig_backward(n, DEV, n, DEV, n, DEV, DEV, DEV, DEV, DEV, n, ctypes.byref(o))
    assert rc == _lib.SCHUR_ERR_WORKSPACE


def test_qz_batched_rejects_each_bad_argument():
    lib = _lib.load()
    b = 2
    n = (ctypes.c_int * b)(N, N)
    ptr = (ctypes.c_void_p * b)(4096, 8192)
    ld = (ctypes.c_int * b)(N, N)
    info = (ctypes.c_int * b)()
    valid = [b, n, ptr, ld, ptr, ld, ptr, ld, ptr, ld, ptr, ptr, ptr, info]
    bad_ld = (ctypes.c_int * b)(N, N - 1)
    bad_n = (ctypes.c_int * b)(N, 0)
    bad_ptr = (ctypes.c_void_p * b)(4096, None)
    cases = {0: [-1], 1: [None, bad_n], 2: [None, bad_ptr], 3: [None, bad_ld], 4: [None, bad_ptr], 5: [None, bad_ld],
             6: [None, bad_ptr], 7: [None, bad_ld], 8: [None, bad_ptr], 9: [None, bad_ld], 10: [None, bad_ptr],
             11: [None, bad_ptr], 12: [None, bad_ptr], 13: [None]}
    for i, bads in cases.items():
        for bad in bads:
            _expect(lib.schur_qz_batched, valid + [_opts()], i, bad)


def test_ht_reduce_batched_rejects_each_bad_argument():
    lib = _lib.load()
    b = 2
    n = (ctypes.c_int * b)(N, N)
    ptr = (ctypes.c_void_p * b)(4096, 8192)
    ld = (ctypes.c_int * b)(N, N)
    info = (ctypes.c_int * b)()
    valid = [b, n, ptr, ld, ptr, ld, ptr, ld, ptr, ld, info]
    bad_ld = (ctypes.c_int * b)(N, N - 1)
    bad_n = (ctypes.c_int * b)(N, 0)
    bad_ptr = (ctypes.c_void_p * b)(4096, None)
    cases = {0: [-1], 1: [None, bad_n], 2: [None, bad_ptr], 3: [None, bad_ld], 4: [None, bad_ptr], 5: [None, bad_ld],
             6: [None, bad_ptr], 7: [None, bad_ld], 8: [None, bad_ptr], 9: [None, bad_ld], 10: [None]}
    for i, bads in cases.items():
        for bad in bads:
            _expect(lib.schur_ht_reduce_batched, valid + [_opts()], i, bad)


def test_factor_backward_batched_rejects_each_bad_argument():
    lib = _lib.load()
    b = 2
    n = (ctypes.c_int * b)(N, N)
    ptr = (ctypes.c_void_p * b)(4096, 8192)
    ld = (ctypes.c_int * b)(N, N)
    valid = [b, n, ptr, ld, ptr, ld, ptr, ld, ptr, ld, ptr, ld]
    bad_ld = (ctypes.c_int * b)(N, N - 1)
    bad_n = (ctypes.c_int * b)(N, 1025)
    bad_ptr = (ctypes.c_void_p * b)(4096, None)
    cases = {0: [-1], 1: [None, bad_n]}
    for i in range(2, 12, 2):
        cases[i] = [None, bad_ptr]
        cases[i + 1] = [None, bad_ld]
    for i, bads in cases.items():
        for bad in bads:
            _expect(lib.schur_factor_backward_batched, valid + [_opts()], i, bad)


def test_short_opts_struct_keeps_defaults_beyond_its_size():
    """An opts block whose struct_size ends before want_z: the library reads
    only struct_size bytes, so want_z keeps its default (1) whatever the
    memory after it holds, and a missing Z / Q is rejected as a bad
    argument, before any device work (every entry point reads opts through
    the same reader)."""
    lib = _lib.load()
    o = _lib.make_opts(0, want_z=0)
    o.struct_size = _lib.SchurOpts.want_z.offset
    ob = ctypes.byref(o)
    assert lib.schur_hessenberg(N, DEV, N, None, N, DEV, DEV, ob) == -4
    assert lib.schur_qz(N, DEV, N, DEV, N, None, N, None, N, DEV, DEV, DEV, ob) == -6
    assert lib.schur_ht_reduce(N, DEV, N, DEV, N, None, N, None, N, ob) == -6


def test_misaligned_or_small_workspace_is_refused():
    """A caller workspace must be 256-byte aligned: a misaligned one (large
    enough) and an aligned one that is too small both return
    SCHUR_ERR_WORKSPACE before any device work, in every entry point that
    takes scratch from opts."""
    lib = _lib.load()
    calls = {
        "schur_eigenvectors": lambda ob: lib.schur_eigenvectors(N, DEV, N, DEV, N, DEV, DEV, DEV, N, ob),
        "schur_hessenberg_reduce": lambda ob: lib.schur_hessenberg_reduce(N, DEV, N, DEV, N, ob),
        "schur_ht_reduce": lambda ob: lib.schur_ht_reduce(N, DEV, N, DEV, N, DEV, N, DEV, N, ob),
        "schur_qz": lambda ob: lib.schur_qz(N, DEV, N, DEV, N, DEV, N, DEV, N, DEV, DEV, DEV, ob),
        "schur_factor_backward": lambda ob: lib.schur_factor_backward(N, DEV, N, DEV, N, DEV, N, DEV, N, DEV, N,
                                                                      ob),
        "schur_eig_backward (per-warp path)": lambda ob: lib.schur_eig_backward(N, DEV, N, DEV, N, DEV, DEV, DEV,
                                                                               DEV, DEV, N, ob),
        "schur_eig_backward (blocked path)": lambda ob: lib.schur_eig_backward(2000, DEV, 2000, DEV, 2000, DEV,
                                                                              DEV, DEV, DEV, DEV, 2000, ob),
    }
    for name, call in calls.items():
        o = _lib.make_opts(0)
        o.workspace = 4096 + 8
        o.workspace_bytes = 1 << 40
        assert call(ctypes.byref(o)) == _lib.SCHUR_ERR_WORKSPACE, name
        o.workspace = 4096
        o.workspace_bytes = 8
        assert call(ctypes.byref(o)) == _lib.SCHUR_ERR_WORKSPACE, name
