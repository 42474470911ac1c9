"""Write the LAPACK eigenvalues of the n = 20000 hess_n benchmark matrix.

Library cross-check (LAPACK dgeev through scipy, OpenBLAS, all host cores) of
the paper's hess_n family (Sec. 5.3 item 3) at the benchmark's order and seed.
The result is an independent eigenvalue multiset for the full-size reduction:
the GPU's eigenvalues at n = 20000 are matched against it.  It takes tens of
minutes on a few cores, so it is run once and stored next to this script:

    python tests/golden/make_hess_n20000_eigvals.py

Output: hess_n20000_seed2023_eigvals.npy (complex128, length 20000, in
LAPACK's order) and a one-line JSON record of how it was made.
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

from paper_2007_03576_gb300 import inputs  # noqa: E402

N, SEED = 20000, 2023


def main():
    H = inputs.hessrand(N, SEED)
    t0 = time.perf_counter()
    w = scipy.linalg.eigvals(H, overwrite_a=True, check_finite=False)
    sec = time.perf_counter() - t0
    out = os.path.join(HERE, f"hess_n{N}_seed{SEED}_eigvals.npy")
    np.save(out, w.astype(np.complex128))
    rec = {"n": N, "seed": SEED, "routine": "scipy.linalg.eigvals (LAPACK dgeev)", "seconds": round(sec, 1),
           "scipy": scipy.__version__, "cores": os.cpu_count(), "machine": platform.machine(),
           "trace_sum_re": float(np.sum(w.real))}
    with open(os.path.join(HERE, f"hess_n{N}_seed{SEED}_eigvals.json"), "w") as f:
        f.write(json.dumps(rec) + "\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
