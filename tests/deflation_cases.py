"""Boundary cases of the deflation tests of Sec. 5.6, shared by the oracle
pins (CPU) and the GPU checks of the device's copies of the tests.

Each case sits on one side of one threshold of a test, with the outcome
fixed by a closed-form eigenvalue perturbation or by the threshold's
definition, stated beside the case."""

import numpy as np

from oracle import qr

U = qr.U


def _block(h11, h12, h21, h22, n=4, k=2, left=0.0, right=0.0):
    """n x n Hessenberg matrix whose rows/columns k-1, k hold [[h11, h12],
    [h21, h22]], with h_{k-1,k-2} = left and h_{k+1,k} = right; zero
    elsewhere, so that only these entries enter the test of H[k, k-1]."""
    H = np.zeros((n, n))
    H[k - 1, k - 1], H[k - 1, k], H[k, k - 1], H[k, k] = h11, h12, h21, h22
    H[k - 1, k - 2] = left
    H[k + 1, k] = right
    return H


# (case, H, expected) with the reason each outcome is fixed:
#  - plain threshold: with h12 = 0 the 2x2 block is triangular whatever h21,
#    so only |h21| <= u (|h11| + |h22|) decides (u (2 + 1) = 3u);
#  - Ahues-Tisseur: with h11 = 2, h22 = h12 = 1, dropping h21 = x moves the
#    eigenvalues by ~ x h12 / (h11 - h22) = x, negligible iff x <= u |h22|;
#    for u < x <= 3u the plain test alone would (wrongly) accept;
#  - equal diagonal, large coupling: [[1, 1], [1e-17, 1]] has eigenvalues
#    1 +- 3.2e-9, so dropping 1e-17 is not negligible although
#    1e-17 <= u (1 + 1);
#  - zero diagonal: the plain test takes |h_{k-1,k-2}| + |h_{k+1,k}| instead;
#  - below nu n / u every entry is negligible;
#  - h22 = 0 at the floor: [[1, 1], [x, 0]] has the eigenvalue ~ -x, and the
#    refinement compares |h21| |h12| / (max(|h22|, |h11 - h22|) +
#    max(|h21|, |h12|)) = x / 2 with the absolute floor nu n / u (x = 1.5 of
#    that floor is negligible, x = 3 of it is not).
SML4 = qr.smlnum(4)
SUBDIAG_CASES = [
    ("plain below", _block(2.0, 0.0, 2.9 * U, 1.0), True),
    ("plain above", _block(2.0, 0.0, 3.1 * U, 1.0), False),
    ("refinement below", _block(2.0, 1.0, 0.9 * U, 1.0), True),
    ("refinement flips", _block(2.0, 1.0, 2.0 * U, 1.0), False),
    ("equal diagonal, coupled", _block(1.0, 1.0, 1e-17, 1.0), False),
    ("equal diagonal, uncoupled", _block(1.0, 0.0, 1e-17, 1.0), True),
    ("zero diagonal, neighbours", _block(0.0, 0.0, 2.9 * U, 0.0, left=1.0, right=2.0), True),
    ("zero diagonal, above", _block(0.0, 0.0, 3.1 * U, 0.0, left=1.0, right=2.0), False),
    ("zero diagonal, no neighbours", _block(0.0, 0.0, 1e-290, 0.0), False),
    ("below nu n / u", _block(0.0, 0.0, 1e-300, 0.0), True),
    ("h22 = 0 at the floor", _block(1.0, 1.0, 1.5 * SML4, 0.0), True),
    ("h22 = 0 above the floor", _block(1.0, 1.0, 3.0 * SML4, 0.0), False),
]


# AED deflation test (Sec. 5.6 item 1, LAPACK-style; items 2-3 norm-stable
# and fixed): records (a, b, c, d, s_j, s_{j-1}, block size), deflation mode,
# threshold, ||H||_F, expected.  1x1 block d = 2: deflatable iff
# |s_j| <= u |d|; 2x2 block [[1, 4], [-1, 1]]: h^ = sqrt|1 * 1| +
# sqrt|4 * -1| = 3, deflatable iff max(|s_j|, |s_{j-1}|) <= u h^; norm-stable
# with ||H||_F = 10: <= 10 u; fixed with threshold 1e-3: <= 1e-3.
HHAT = 3.0
SPIKE_CASES = [
    ("1x1 below", (0, 0, 0, 2.0, 0.5 * U * 2.0, 0.0, 1), "lapack", 0.0, 1.0, True),
    ("1x1 above", (0, 0, 0, 2.0, 2.0 * U * 2.0, 0.0, 1), "lapack", 0.0, 1.0, False),
    ("2x2 below", (1.0, 4.0, -1.0, 1.0, 0.5 * U * HHAT, 0.9 * U * HHAT, 2), "lapack", 0.0, 1.0, True),
    ("2x2 above (upper row)", (1.0, 4.0, -1.0, 1.0, 0.0, 1.1 * U * HHAT, 2), "lapack", 0.0, 1.0, False),
    ("2x2 above (lower row)", (1.0, 4.0, -1.0, 1.0, 1.1 * U * HHAT, 0.0, 2), "lapack", 0.0, 1.0, False),
    ("1x1 at nu n / u", (0, 0, 0, 0.0, 0.5 * qr.smlnum(4), 0.0, 1), "lapack", 0.0, 1.0, True),
    ("norm below", (0, 0, 0, 2.0, 9 * U, 0.0, 1), "norm", 0.0, 10.0, True),
    ("norm above", (0, 0, 0, 2.0, 11 * U, 0.0, 1), "norm", 0.0, 10.0, False),
    ("fixed below", (1.0, 4.0, -1.0, 1.0, 9e-4, 9e-4, 2), "fixed", 1e-3, 1.0, True),
    ("fixed above", (1.0, 4.0, -1.0, 1.0, 9e-4, 2e-3, 2), "fixed", 1e-3, 1.0, False),
]


def spike_case_args(rec, mode, thold, normh, n=4):
    """The oracle's arguments (T, spike, j, bs, Params, n) for one record."""
    a, b, c, d, sj, sjm1, bs = rec
    if bs == 1:
        T = np.array([[d]])
        return T, np.array([sj]), 0, 1, qr.Params(deflation=mode, thold=thold, normH=normh), n
    T = np.array([[a, b], [c, d]])
    return T, np.array([sjm1, sj]), 1, 2, qr.Params(deflation=mode, thold=thold, normH=normh), n
