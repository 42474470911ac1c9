"""The pipelined order of the AED deflation checks and swaps (the order the
CUDA path runs, see the AED kernel) computes what the sequential order of
Sec. 2.5 computes, up to rounding.

Sequential order (the oracle's ``aed``): test the bottom unevaluated block;
a block that fails is moved by adjacent swaps to just below the blocks that
failed before it, then the next bottom block is tested.

Pipelined order: in every round each failed block that has an unevaluated
block directly above it swaps with that block, and the bottom block is
tested when it is unevaluated.  A failed block's later swaps act above the
blocks still to be tested, and swaps of disjoint adjacent pairs commute, so
both orders perform the same swaps and the same tests.

The pipelined schedule is written here with the oracle's own swap and
deflation test, run on the oracle's window Schur form, and compared with
``oracle.qr.aed``: the same number of deflated eigenvalues, the same
candidates (to rounding), and an orthogonal similarity of the window.
"""

import numpy as np
import pytest

from oracle import metrics, qr
from paper_2007_03576_gb300 import inputs


def _blocks(T, lo, hi):
    out, j = [], lo
    while j < hi:
        b = 2 if j + 1 < hi and T[j + 1, j] != 0.0 else 1
        out.append(b)
        j += b
    return out


def _pipelined(T, V, s, info, P, n):
    """Pipelined checks and swaps on rows [info, nw) of the window T (Schur
    form, transform V); returns (ns, failed, rounds)."""
    nw = T.shape[0]
    size = _blocks(T, info, nw)
    state = ["u"] * len(size)  # "u" not yet tested, "f" failed
    ns = nw
    failed = False
    rounds = 0
    for rounds in range(1, 4 * nw + 16):
        pairs = [k for k in range(1, len(size)) if state[k] == "f" and state[k - 1] == "u"]
        check = bool(size) and state[-1] == "u"
        if not pairs and not check:
            break
        pos = np.concatenate([[info], info + np.cumsum(size)]).astype(int)
        # the bottom block is not part of any pair: its test reads nothing
        # the swaps of this round change
        if check:
            bs = size[-1]
            if qr.spike_deflatable(T, s * V[0, :], ns - 1, bs, P, n):
                ns -= bs
                size.pop()
                state.pop()
            else:
                state[-1] = "f"
        for k in pairs:
            j, p, q = int(pos[k - 1]), size[k - 1], size[k]
            if not qr.swap_adjacent(T, V, j, p, q):
                failed = True
                continue
            size[k - 1], size[k] = q, p
            state[k - 1], state[k] = "f", "u"
        if failed:
            break
    return ns, failed, rounds


def _window_case(n, nw, pre, seed, npairs=4):
    """hess_n matrix after `pre` multishift sweeps whose shifts are the
    eigenvalues of the trailing 2*npairs block: the bottom starts to converge,
    so an AED both deflates and reorders."""
    H = inputs.hessrand(n, seed)
    Z = np.eye(n)
    for _ in range(pre):
        lam = np.linalg.eigvals(H[n - 2 * npairs:, n - 2 * npairs:])
        pairs = qr.pairs_from_candidates([(z.real, z.imag) for z in lam], npairs)
        qr.multishift_sweep(H, Z, 0, n - 1, pairs)
    return H


@pytest.mark.parametrize("n,nw,pre,seed", [(120, 40, 4, 11), (200, 64, 6, 12), (260, 96, 6, 11)])
def test_pipelined_order_matches_sequential_aed(n, nw, pre, seed):
    H = _window_case(n, nw, pre, seed)
    # the window's Schur form by double-shift QR on both sides (crossover
    # above nw), so that both orders start from the same T and V
    P = qr.Params(normH=np.linalg.norm(H), nwin_francis=max(nw, 75))
    kbot = n - 1
    kwtop = kbot - nw + 1
    s = H[kwtop, kwtop - 1]
    # sequential: the oracle's AED step itself
    Hs, Zs = H.copy(), np.eye(n)
    nd_seq, cand_seq = qr.aed(Hs, Zs, 0, kbot, nw, P)
    # pipelined: same window Schur form, then the pipelined schedule
    T0 = np.triu(H[kwtop:, kwtop:], -1).copy()
    T, V = T0.copy(), np.eye(nw)
    info = qr.francis_qr(T, V, 0, nw - 1, P.for_window(), nw)
    ns, failed, rounds = _pipelined(T, V, s, info, P, n)
    nd_pipe = nw - ns
    assert not failed
    assert nd_pipe == nd_seq
    assert nd_seq > 0  # the case exercises both deflation and reordering
    cand_pipe = qr.block_eigs(T, info, ns)
    assert len(cand_pipe) == len(cand_seq)
    lam_p = np.array([complex(*c) for c in cand_pipe])
    lam_s = np.array([complex(*c) for c in cand_seq])
    _, dist = metrics.match_eigenvalues(lam_s, lam_p)
    assert np.max(dist) <= 1e-10 * np.linalg.norm(H)
    # the failed candidates keep the sequential order (top to bottom), so the
    # candidate lists agree entry by entry, not only as multisets
    assert np.max(np.abs(lam_p - lam_s)) <= 1e-8 * np.linalg.norm(H)
    # orthogonal similarity of the window, Schur form kept
    assert np.linalg.norm(V @ T @ V.T - T0) <= 1e-13 * np.linalg.norm(T0) * nw
    assert np.linalg.norm(V.T @ V - np.eye(nw)) <= 1e-13 * nw
    assert np.max(np.abs(np.tril(T, -2))) == 0.0
    # far fewer rounds than sequential swaps: the point of the pipeline
    assert rounds <= 3 * len(_blocks(T0, 0, nw)) + 4
