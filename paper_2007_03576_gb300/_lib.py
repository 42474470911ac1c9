"""ctypes binding of libschur_gb300.so (argument marshalling only).

The library is built in-tree by ``paper_2007_03576_gb300.build``.  There is no
fallback: if the library cannot be built or loaded, ``load()`` raises.
"""

import ctypes
import os
import re

from . import build as _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "schur_gb300.h")

c_int = ctypes.c_int
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
c_size_t = ctypes.c_size_t
P = ctypes.POINTER

SCHUR_OK = 0
SCHUR_ERR_NONFINITE = -1001
SCHUR_ERR_CUDA = -1002
SCHUR_ERR_NOMEM = -1003
SCHUR_ERR_WORKSPACE = -1004
SCHUR_ERR_UNSUPPORTED = -1005
SCHUR_ERR_TOO_LARGE = -1006

DEFLATION = {"lapack": 0, "norm": 1, "fixed": 2}


class SchurOpts(ctypes.Structure):
    _fields_ = [
        ("struct_size", c_int),
        ("n_shifts", c_int),
        ("aed_window", c_int),
        ("bulges_per_chain", c_int),
        ("nmin", c_int),
        ("nibble", c_int),
        ("deflation", c_int),
        ("fixed_thold", c_double),
        ("want_z", c_int),
        ("z_init", c_int),
        ("stream", c_void_p),
        ("workspace", c_void_p),
        ("workspace_bytes", c_size_t),
        ("timing", c_int),
        ("nmin_window", c_int),
        ("recompute_shifts", c_int),
        ("split_products", c_int),
    ]


class SchurStats(ctypes.Structure):
    _fields_ = [
        ("aed_steps", c_int),
        ("sweeps", c_int),
        ("small_qr", c_int),
        ("deflated_by_aed", c_int),
        ("window_launches", c_int),
        ("sweep_gemm_flops", c_double),
        ("aed_gemm_flops", c_double),
        ("reflector_flops", c_double),
        ("update_launches", c_int),
        ("chase_launches", c_int),
        ("t_chase_ms", c_double),
        ("t_update_ms", c_double),
        ("t_aed_ms", c_double),
        ("t_aed_update_ms", c_double),
        ("t_small_ms", c_double),
        ("aed_cycles_schur", c_double),
        ("aed_cycles_post", c_double),
        ("kernel_launches", ctypes.c_longlong),
        ("t_z_ms", c_double),
        ("graph_built", c_int),
        ("shift_recomputations", c_int),
        ("flops", c_double),
    ]


_SIGS = {
    "schur_default_opts": (c_int, [P(SchurOpts)]),
    "schur_status_string": (ctypes.c_char_p, [c_int]),
    "schur_workspace_size": (c_int, [c_int, P(SchurOpts), P(c_size_t)]),
    "schur_hessenberg": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, P(SchurOpts)]),
    "schur_last_stats": (c_int, [P(SchurStats)]),
    "schur_last_error_detail": (ctypes.c_char_p, []),
    "schur_hessenberg_batched": (c_int, [c_int, P(c_int), P(c_void_p), P(c_int), P(c_void_p), P(c_int),
                                         P(c_void_p), P(c_void_p), P(c_int), P(SchurOpts)]),
    "schur_eig_backward_workspace": (c_int, [c_int, P(c_size_t)]),
    "schur_eig_backward": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_int, P(SchurOpts)]),
    "schur_eig_backward_batched": (c_int, [c_int, P(c_int), P(c_void_p), P(c_int), P(c_void_p), P(c_int),
                                           P(c_void_p), P(c_void_p), P(c_void_p), P(c_void_p), P(c_void_p),
                                           P(c_int), P(SchurOpts)]),
    "schur_sweep": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_int, c_int, P(c_double), c_int, c_int,
                            P(SchurOpts)]),
    "schur_aed": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_int, P(c_int), P(c_double),
                          P(c_double), P(c_int), P(SchurOpts)]),
    "schur_small_qr": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_int, c_int, P(SchurOpts)]),
    "schur_apply_u": (c_int, [c_int, c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_int,
                              P(SchurOpts)]),
    "schur_fastmath_eval": (c_int, [c_int, c_void_p, c_void_p, P(SchurOpts)]),
    "schur_batched_set_table": (c_int, [c_int, P(c_int), P(c_int), P(c_int)]),
    "schur_hessenberg_noalloc": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p,
                                         P(SchurOpts)]),
    "schur_fp64_fma_probe": (c_int, [c_int, c_int, c_void_p, P(c_double), P(SchurOpts)]),
    "schur_hessenberg_reduce": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, P(SchurOpts)]),
    "schur_hessenberg_reduce_workspace": (c_int, [c_int, P(c_size_t)]),
    "schur_eigenvectors": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int,
                                   P(SchurOpts)]),
    "schur_eigenvectors_workspace": (c_int, [c_int, c_int, P(c_size_t)]),
    "schur_ht_reduce": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int,
                                P(SchurOpts)]),
    "schur_ht_reduce_batched": (c_int, [c_int, P(c_int), P(c_void_p), P(c_int), P(c_void_p), P(c_int),
                                        P(c_void_p), P(c_int), P(c_void_p), P(c_int), P(c_int), P(SchurOpts)]),
    "schur_qz": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p,
                         c_void_p, c_void_p, P(SchurOpts)]),
    "schur_factor_backward": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int,
                                      c_void_p, c_int, P(SchurOpts)]),
    "schur_factor_backward_batched": (c_int, [c_int, P(c_int), P(c_void_p), P(c_int), P(c_void_p), P(c_int),
                                              P(c_void_p), P(c_int), P(c_void_p), P(c_int), P(c_void_p), P(c_int),
                                              P(SchurOpts)]),
    "schur_sweep_split_tasks": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, P(c_int), P(c_int)]),
    "schur_qz_sweep": (c_int, [c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_int,
                               c_int, c_double, c_double, P(SchurOpts)]),
    "schur_qz_batched": (c_int, [c_int, P(c_int), P(c_void_p), P(c_int), P(c_void_p), P(c_int), P(c_void_p),
                                 P(c_int), P(c_void_p), P(c_int), P(c_void_p), P(c_void_p), P(c_void_p), P(c_int),
                                 P(SchurOpts)]),
    "schur_chase_schedule": (c_int, [c_int, c_int, c_int, c_int, c_int, c_void_p, P(c_int), P(c_int), P(c_int)]),
    "schur_vigilant_eval": (c_int, [c_int, c_void_p, c_int, c_double, c_double, c_int, c_void_p, P(SchurOpts)]),
    "schur_spike_eval": (c_int, [c_int, c_void_p, c_int, c_double, c_double, c_int, c_void_p, P(SchurOpts)]),
}

_LIB = None


def header_functions():
    """Names of the functions declared in include/schur_gb300.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(schur_\w+)\s*\(", txt, flags=re.M)))


def load(build=True):
    """Build (if stale) and load the library; raises on failure."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libschur_gb300.so not found at {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def make_opts(stream=0, **kw):
    """schur_opts with the library defaults, overridden by keyword args
    (deflation may be "lapack" / "norm" / "fixed")."""
    lib = load()
    o = SchurOpts()
    lib.schur_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "deflation" and isinstance(v, str):
            v = DEFLATION[v]
        setattr(o, k, v)
    o.stream = stream
    return o


def status(code):
    s = load().schur_status_string(int(code)).decode()
    if int(code) == SCHUR_ERR_CUDA:
        s += ": " + load().schur_last_error_detail().decode()
    return s
