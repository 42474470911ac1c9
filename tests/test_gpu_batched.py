"""Batched path (one persistent launch over many matrices) vs the oracle and
vs the single-matrix path.  Same tolerances as test_gpu_parity: backward
error and orthogonality <= 1e-13, standardised structure, eigenvalues within
1e-10 * kappa_i * ||H||_F of the oracle's."""

import math

import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")

from oracle import qr, metrics  # noqa: E402
from paper_2007_03576_gb300 import api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


def _check(H, S, Z):
    n = H.shape[0]
    nh = max(np.linalg.norm(H), 1e-300)
    assert np.linalg.norm(Z @ S @ Z.T - H) / nh <= 1e-13
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) / math.sqrt(n) <= 1e-13
    assert metrics.schur_structure_errors(S) == []


def test_batched_mixed_sizes_vs_oracle():
    sizes = [1, 2, 3, 5, 17, 40, 76, 90, 120, 150, 33, 8, 64, 101]
    Hs = [inputs.hessrand(n, [77, i]) for i, n in enumerate(sizes)]
    S, Z, wr, wi, info = api.schur_batched([_dev(h) for h in Hs])
    assert info == [0] * len(sizes)
    for h, s, z, a, b in zip(Hs, S, Z, wr, wi):
        Sg, Zg = s.cpu().numpy(), z.cpu().numpy()
        _check(h, Sg, Zg)
        So, Zo, wro, wio, _ = qr.schur(h)
        _, kap = metrics.eig_condition(So)
        perm, dist = metrics.match_eigenvalues(wro + 1j * wio, a.cpu().numpy() + 1j * b.cpu().numpy())
        assert np.all(dist <= 1e-10 * kap * np.linalg.norm(h))


def test_batched_large_members_invariants():
    """Members up to the workload's largest size (768): residual,
    orthogonality, structure and the trace invariants; the eigenvalues
    against LAPACK's dgeev (library cross-check, scipy) within
    1e-10 kappa_i ||H||_F, kappa_i from LAPACK's left and right vectors, and
    the 300-row member against the oracle as well."""
    sizes = [768, 500, 300, 640, 200]
    Hs = [inputs.hessrand(n, [5, i]) for i, n in enumerate(sizes)]
    S, Z, wr, wi, info = api.schur_batched([_dev(h) for h in Hs])
    assert info == [0] * len(sizes)
    for h, s, z, a, b in zip(Hs, S, Z, wr, wi):
        _check(h, s.cpu().numpy(), z.cpu().numpy())
        lam = a.cpu().numpy() + 1j * b.cpu().numpy()
        n = h.shape[0]
        nh = np.linalg.norm(h)
        assert abs(np.sum(lam) - np.trace(h)) < 1e-12 * n * nh
        assert abs(np.sum(lam ** 2) - np.trace(h @ h)) < 1e-12 * n * nh ** 2
        w, vl, vr = scipy.linalg.eig(h, left=True, right=True)
        kap = np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0) / np.abs(np.sum(np.conj(vl) * vr, axis=0))
        perm, dist = metrics.match_eigenvalues(w, lam)
        assert np.all(dist <= 1e-10 * kap * nh), float(np.max(dist / (kap * nh)))
        if n == 300:
            So, Zo, wro, wio, _ = qr.schur(h)
            _, kap_o = metrics.eig_condition(So)
            perm, dist = metrics.match_eigenvalues(wro + 1j * wio, lam)
            assert np.all(dist <= 1e-10 * kap_o * nh)


def test_batched_matches_single_path():
    """The batched engine and the single-matrix (windowed) path reduce the
    same matrix to the same spectrum."""
    Hs = [inputs.hessrand(n, [9, n]) for n in (130, 260)]
    S, Z, wr, wi, info = api.schur_batched([_dev(h) for h in Hs])
    for h, a, b in zip(Hs, wr, wi):
        S1, Z1, wr1, wi1, rc = api.schur(_dev(h))
        S1n = S1.cpu().numpy()
        _, kap = metrics.eig_condition(S1n)
        perm, dist = metrics.match_eigenvalues(wr1.cpu().numpy() + 1j * wi1.cpu().numpy(),
                                               a.cpu().numpy() + 1j * b.cpu().numpy())
        assert np.all(dist <= 1e-10 * kap * np.linalg.norm(h))


def test_batched_table_and_zinit():
    """A custom bucket table and accumulation into given Z (z_init = 1)."""
    api.set_batched_table([100, 10 ** 6], [4, 16], [16, 48])
    try:
        H = inputs.hessrand(180, 3)
        Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((180, 180)))
        Hc = _dev(H).clone()
        Zc = _dev(Q).clone()
        wr = torch.empty(180, dtype=torch.float64, device="cuda")
        wi = torch.empty_like(wr)
        info = api.schur_batched_inplace([Hc], [Zc], [wr], [wi], z_init=1)
        assert info == [0]
        _check(Q @ H @ Q.T, Hc.cpu().numpy(), Zc.cpu().numpy())
    finally:
        api.set_batched_table([], [], [])
    with pytest.raises(RuntimeError):
        api.set_batched_table([10], [1], [16])


def test_batched_graph_is_replayed_for_the_same_shape():
    """The captured graph is cached per batch shape: a second call with the
    same shape replays it with the new matrices' descriptors (and is just as
    correct); a different batch size captures a new one.  The kernel's
    counted algorithmic flops are reported."""
    sizes = [90, 140, 60]
    results = []
    for call, seed in enumerate((41, 42)):
        Hs = [inputs.hessrand(n, [seed, b]) for b, n in enumerate(sizes)]
        S, Z, wr, wi, info = api.schur_batched([_dev(h) for h in Hs])
        st = api.last_stats()
        results.append(st["graph_built"])
        assert all(i == 0 for i in info)
        for h, s_, z_ in zip(Hs, S, Z):
            _check(h, s_.cpu().numpy(), z_.cpu().numpy())
        # the work of the iteration on these orders, with Z: of the order of
        # 10-40 n^3 per matrix
        work = sum(n ** 3 for n in sizes)
        assert 2 * work < st["reflector_flops"] < 80 * work, st["reflector_flops"] / work
    assert results[1] == 0
    S, Z, wr, wi, info = api.schur_batched([_dev(inputs.hessrand(50, 43))])
    assert api.last_stats()["graph_built"] == 1 and info == [0]
