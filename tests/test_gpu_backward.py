"""Eigenvalue adjoint (backward) on the GPU vs the oracle's adjoint, closed
forms and central finite differences.  Orders up to 1024 take the per-warp
vector path, larger single matrices the blocked one (compared with the
oracle just above the crossover here, and with closed forms at n = 4096 in
test_gpu_workloads_large).

The adjoint of eigenvalue i scales with its condition number; parity with
the oracle is asserted entrywise on the same Schur factor (both evaluate
dH = Z Re(sum conj(g)/c w x^T) Z^T) within 1e-10 * max_i kappa_i * ||g||."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint, metrics  # noqa: E402
from paper_2007_03576_gb300 import api, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda().t()


@pytest.mark.parametrize("n", [2, 7, 50, 130, 700, 1030])
def test_backward_matches_oracle_adjoint(n):
    H = inputs.hessrand(n, 600 + n)
    S, Z, wr, wi, info = api.schur(_dev(H))
    assert info == 0
    gr, gi = 2 * wr, 2 * wi       # L = sum |lambda|^2
    dH = api.eig_backward(S, Z, wr, wi, gr, gi).cpu().numpy()
    Sn, Zn = S.cpu().numpy(), Z.cpu().numpy()
    ref = adjoint.eig_adjoint(Sn, Zn, gr.cpu().numpy(), gi.cpu().numpy())
    _, kap = metrics.eig_condition(Sn)
    scale = np.max(kap) * np.linalg.norm(np.concatenate([gr.cpu().numpy(), gi.cpu().numpy()]))
    assert np.max(np.abs(dH - ref)) <= 1e-10 * scale, np.max(np.abs(dH - ref)) / scale


def test_backward_closed_forms():
    """g = 1 -> dH = I (sum lambda = tr H); g = 2 conj(lambda) -> dH = 2 H^T
    (sum Re lambda^2 = tr H^2)."""
    n = 60
    H = inputs.hessrand(n, 21)
    S, Z, wr, wi, info = api.schur(_dev(H))
    one = torch.ones(n, dtype=torch.float64, device="cuda")
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    dH = api.eig_backward(S, Z, wr, wi, one, zero).cpu().numpy()
    assert np.max(np.abs(dH - np.eye(n))) < 1e-10
    dH = api.eig_backward(S, Z, wr, wi, 2 * wr, -2 * wi).cpu().numpy()
    assert np.max(np.abs(dH - 2 * H.T)) < 1e-9 * np.linalg.norm(H)


def test_backward_finite_difference_via_autograd():
    """Central differences at h = 1e-6 of L = sum |lambda|^2 (the
    differentiation workload's loss), forward through the GPU, along random
    Hessenberg-pattern directions, against the autograd gradient."""
    n = 40
    H = inputs.hessrand(n, 33)
    Ht = _dev(H).requires_grad_(True)
    wr, wi = api.eigvals(Ht)
    L = (wr * wr + wi * wi).sum()
    (g,) = torch.autograd.grad(L, Ht)
    g = g.cpu().numpy()
    rng = np.random.default_rng(1)

    def loss(M):
        _, _, a, b, _ = api.schur(_dev(M))
        return float((a * a + b * b).sum())

    for _ in range(3):
        E = np.triu(rng.standard_normal((n, n)), -1)
        h = 1e-6
        fd = (loss(H + h * E) - loss(H - h * E)) / (2 * h)
        an = float(np.sum(g * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_backward_batched_matches_single():
    sizes = [64, 100, 37, 150]
    Hs = [inputs.hessrand(n, [40, n]) for n in sizes]
    S, Z, wr, wi, info = api.schur_batched([_dev(h) for h in Hs])
    gr = [2 * a for a in wr]
    gi = [2 * b for b in wi]
    dHs = api.eig_backward_batched(S, Z, wr, wi, gr, gi)
    for s, z, a, b, c, d, dh in zip(S, Z, wr, wi, gr, gi, dHs):
        one = api.eig_backward(s, z, a, b, c, d)
        assert torch.max(torch.abs(one - dh)).item() <= 1e-12 * max(1.0, torch.max(torch.abs(one)).item())

