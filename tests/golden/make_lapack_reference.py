"""Write LAPACK reference spectra for the n = 4096 workloads.

Library cross-check (LAPACK dgeev through scipy, OpenBLAS, host cores) of
the paper's synthetic families (Sec. 5.3) at the orders where the CPU oracle
does not finish in test time:

    python tests/golden/make_lapack_reference.py hessrand 4096 2021
    python tests/golden/make_lapack_reference.py prescribed_nonnormal 4096 2022

hessrand: the eigenvalues of hess_n (Sec. 5.3 item 3) and their condition
numbers kappa_i = ||x_i|| ||y_i|| / |y_i^H x_i| from LAPACK's left and right
eigenvectors.
prescribed_nonnormal: the condition numbers of the block upper triangular
T = D + N whose orthogonal similarity the workload reduces (the eigenvalues
are T's diagonal blocks, known exactly; condition numbers do not change
under an orthogonal similarity).

Output: lapack_<family>_n<N>_seed<SEED>.npz (arrays eig, kappa) and a JSON
line describing the run, next to this script.
"""

import json
import os
import platform
import sys
import time

import numpy as np
import scipy
import scipy.linalg

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import testmats  # noqa: E402
from paper_2007_03576_gb300 import inputs  # noqa: E402


def condition(A):
    w, vl, vr = scipy.linalg.eig(A, left=True, right=True, check_finite=False)
    c = np.abs(np.sum(np.conj(vl) * vr, axis=0))
    kappa = np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0) / np.maximum(c, 1e-300)
    return w, kappa


def main(family, n, seed):
    t0 = time.perf_counter()
    if family == "hessrand":
        w, kappa = condition(inputs.hessrand(n, seed))
    elif family == "prescribed_nonnormal":
        T, lam = testmats.prescribed_blocks(n, np.random.default_rng(seed), nonnormal=True)
        w, kappa = condition(T)
    else:
        raise SystemExit(f"unknown family {family}")
    sec = time.perf_counter() - t0
    stem = f"lapack_{family}_n{n}_seed{seed}"
    np.savez(os.path.join(HERE, stem + ".npz"), eig=w.astype(np.complex128), kappa=kappa)
    rec = {"family": family, "n": n, "seed": seed, "routine": "scipy.linalg.eig (LAPACK dgeev, left+right)",
           "seconds": round(sec, 1), "scipy": scipy.__version__, "cores": os.cpu_count(),
           "machine": platform.machine(), "kappa_max": float(np.max(kappa))}
    with open(os.path.join(HERE, stem + ".json"), "w") as f:
        f.write(json.dumps(rec) + "\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]), int(sys.argv[3]))
