"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every function declared in
include/schur_gb300.h; default options and status strings."""

import ctypes

from paper_2007_03576_gb300 import _lib


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    declared = _lib.header_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
        assert name in _lib._SIGS, f"binding lacks {name}"


def test_default_opts_and_status_strings():
    lib = _lib.load()
    o = _lib.SchurOpts()
    assert lib.schur_default_opts(ctypes.byref(o)) == 0
    assert o.struct_size == ctypes.sizeof(_lib.SchurOpts)
    assert o.nmin == 75 and o.nibble == 14 and o.want_z == 1 and o.deflation == 0
    assert _lib.status(0) == "success"
    assert "NaN" in _lib.status(_lib.SCHUR_ERR_NONFINITE)
    assert "invalid" in _lib.status(-3)
    assert "iteration limit" in _lib.status(7)


def test_workspace_size_grows_with_n():
    lib = _lib.load()
    o = _lib.make_opts(0)
    sizes = []
    for n in (10, 256, 4096, 20000):
        b = ctypes.c_size_t(0)
        assert lib.schur_workspace_size(n, ctypes.byref(o), ctypes.byref(b)) == 0
        sizes.append(b.value)
    assert sizes == sorted(sizes)
    assert sizes[-1] < 512 * 2 ** 20  # scratch is small next to H and Z
    assert lib.schur_workspace_size(-1, ctypes.byref(o), ctypes.byref(ctypes.c_size_t())) == -1


def test_struct_size_zero_reads_the_whole_opts_block():
    """struct_size <= 0 means the whole struct in every entry point: the
    shift and window overrides of such a block change the workspace size
    exactly as those of a block with struct_size = sizeof(schur_opts)."""
    lib = _lib.load()
    full = _lib.make_opts(0, n_shifts=64, aed_window=200)
    zero = _lib.make_opts(0, n_shifts=64, aed_window=200)
    zero.struct_size = 0
    plain = _lib.make_opts(0)
    got = {}
    for name, o in (("full", full), ("zero", zero), ("plain", plain)):
        b = ctypes.c_size_t(0)
        assert lib.schur_workspace_size(20000, ctypes.byref(o), ctypes.byref(b)) == 0
        got[name] = b.value
    assert got["zero"] == got["full"]
    assert got["zero"] != got["plain"]


def test_argument_validation_without_gpu():
    """Invalid arguments are rejected before any device work."""
    lib = _lib.load()
    o = _lib.make_opts(0)
    assert lib.schur_hessenberg(-1, None, 1, None, 1, None, None, ctypes.byref(o)) == -1
    assert lib.schur_hessenberg(4, None, 4, None, 4, None, None, ctypes.byref(o)) == -2
    assert lib.schur_hessenberg(4, 1, 3, None, 4, None, None, ctypes.byref(o)) == -3
    assert lib.schur_hessenberg(0, None, 1, None, 1, None, None, ctypes.byref(o)) == 0
    assert lib.schur_apply_u(2, None, 1, 0, 0, 1, 1, None, 1, ctypes.byref(o)) == -1
