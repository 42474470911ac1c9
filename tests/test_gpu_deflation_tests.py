"""The device's copies of the deflation tests of Sec. 5.6 (vigilant test of a
subdiagonal entry, AED spike test) on the boundary cases that pin the
oracle's tests, through the C ABI: the device takes the same decision as the
oracle and as the case's stated outcome on every case."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from deflation_cases import SPIKE_CASES, SUBDIAG_CASES, spike_case_args  # noqa: E402
from oracle import qr  # noqa: E402
from paper_2007_03576_gb300 import _lib  # noqa: E402

pytestmark = pytest.mark.gpu

MODES = {"lapack": 0, "norm": 1, "fixed": 2}


def test_vigilant_test_matches_oracle_on_boundary_cases():
    Hs = np.stack([np.asarray(H, dtype=np.float64).T.copy() for _, H, _ in SUBDIAG_CASES])  # column-major 4x4
    Hd = torch.from_numpy(Hs.reshape(-1)).cuda()
    out = torch.full((len(SUBDIAG_CASES),), -1, dtype=torch.int32, device="cuda")
    rc = _lib.load().schur_vigilant_eval(len(SUBDIAG_CASES), Hd.data_ptr(), 0, 0.0, 1.0, 4, out.data_ptr(),
                                         ctypes.byref(_lib.make_opts(0)))
    assert rc == 0, _lib.status(rc)
    got = out.cpu().numpy()
    for (name, H, expected), g in zip(SUBDIAG_CASES, got):
        oracle = bool(qr.subdiag_negligible(H, 2, 0, 3, qr.Params(), 4))
        assert bool(g) == oracle == expected, name


@pytest.mark.parametrize("mode", ["lapack", "norm", "fixed"])
def test_spike_test_matches_oracle_on_boundary_cases(mode):
    cases = [c for c in SPIKE_CASES if c[2] == mode]
    thold, normh = cases[0][3], cases[0][4]
    recs = np.array([list(c[1]) for c in cases], dtype=np.float64)
    rd = torch.from_numpy(recs.reshape(-1)).cuda()
    out = torch.full((len(cases),), -1, dtype=torch.int32, device="cuda")
    rc = _lib.load().schur_spike_eval(len(cases), rd.data_ptr(), MODES[mode], thold, normh, 4, out.data_ptr(),
                                      ctypes.byref(_lib.make_opts(0)))
    assert rc == 0, _lib.status(rc)
    for (name, rec, m, th, nh, expected), g in zip(cases, out.cpu().numpy()):
        oracle = bool(qr.spike_deflatable(*spike_case_args(rec, m, th, nh)))
        assert bool(g) == oracle == expected, name
