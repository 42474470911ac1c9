"""Plain, slow CPU FP64 oracle for the Hessenberg -> real Schur reduction.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path (``paper_2007_03576_gb300/csrc``): the two are written separately
from the paper and compared on the same seeded inputs.

Every routine is written in numpy float64, one reflector / rotation at a time,
in the order the paper describes (Myllykoski, "Algorithm 1019: A task-based
multi-shift QR/QZ algorithm with aggressive early deflation", ACM TOMS 2021):

* ``householder``  -- reflectors and the Householder Hessenberg reduction
                      (Sec. 1 phase (i); used for input generation, and for the
                      spike elimination of Sec. 2.5 step 3).
* ``qr``           -- Francis double-shift sweep (Sec. 2.2, Fig. 1), the
                      small-bulge multishift sweep (Sec. 2.3, Fig. 2), the
                      deflation conditions (Sec. 5.6), eigenvalue reordering
                      (Sec. 2.5 step 2), AED (Sec. 2.5, Fig. 4) and the
                      iterative driver (Sec. 2.1).
* ``metrics``      -- the accuracy metrics of Sec. 5.4, eigenvectors of the
                      quasi-triangular Schur factor and eigenvalue condition
                      numbers.
* ``adjoint``      -- the eigenvalue adjoint dH (not in the paper; first-order
                      eigenvalue perturbation theory).
* ``testmats``     -- matrices with known spectra (Sec. 5.3 syn_n, companion,
                      cyclic, prescribed spectrum).
* ``qz``           -- the generalized case of the paper's remarks: the
                      Hessenberg-triangular reduction, double-shift QZ sweeps,
                      infinite eigenvalues chased to the top of the active
                      block, standardised 2x2 blocks.

Parity pins (what fixes each function independently of itself) live in
``tests/test_oracle_*.py``.  Functions with no independent pin say
"parity unpinned" in their docstring.
"""

from . import householder, qr, metrics, adjoint, testmats, qz  # noqa: F401
