"""Autotuner for the batched path's per-size-bucket (shifts, AED window) table.

For every size bucket a sample batch (one wave: as many matrices as the GPU
has SMs, sizes uniform within the bucket, hess_n entries) is reduced with each
candidate pair, timed with CUDA events; the fastest candidate is kept and the
resulting table installed with ``schur_batched_set_table``.  Only timing
decides; every candidate computes the same reduction (same deflation rules),
so the choice does not change what is computed, only how fast.
"""

import json

import numpy as np
import torch

from . import api, inputs

BUCKETS = [149, 299, 589, 1024]
NMIN_CANDIDATES = [48, 75, 100]
CANDIDATES = {
    149: [(4, 16), (8, 24), (8, 32)],
    299: [(8, 24), (8, 32), (16, 48)],
    589: [(8, 32), (16, 48), (32, 64)],
    1024: [(16, 48), (32, 64), (48, 96), (64, 128)],
}


def _time_batch(Hs, table, reps=1):
    api.set_batched_table(*table)
    best = None
    for _ in range(reps):
        Ss = [h.clone() for h in Hs]
        Zs = [api.new_colmajor(h.shape[0]) for h in Hs]
        wrs = [torch.empty(h.shape[0], dtype=torch.float64, device="cuda") for h in Hs]
        wis = [torch.empty_like(w) for w in wrs]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        info = api.schur_batched_inplace(Ss, Zs, wrs, wis)
        e1.record()
        torch.cuda.synchronize()
        if any(info):
            return float("inf")
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    return best


def autotune_batched(lo=32, hi=768, seed=7, per_bucket=None, verbose=False):
    """Tune the bucket table for sizes in [lo, hi]; returns
    {"max_n": [...], "ns": [...], "nw": [...], "timings": {...}} and installs
    the table."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_bucket = per_bucket or sms
    rng = np.random.default_rng(seed)
    chosen_ns, chosen_nw, timings = [], [], {}
    prev = lo - 1
    # buckets are tuned one at a time with the other buckets at their
    # current choice (or the first candidate)
    for bmax in BUCKETS:
        blo, bhi = max(lo, prev + 1), min(hi, bmax)
        prev = bmax
        if blo > bhi:
            chosen_ns.append(CANDIDATES[bmax][0][0])
            chosen_nw.append(CANDIDATES[bmax][0][1])
            continue
        sizes = rng.integers(blo, bhi + 1, size=per_bucket)
        Hs = []
        for i, n in enumerate(sizes):
            H = inputs.hessrand(int(n), [seed, bmax, i])
            Hs.append(torch.from_numpy(np.ascontiguousarray(H.T)).cuda().t())
        res = []
        for ns, nw in CANDIDATES[bmax]:
            k = len(chosen_ns)
            tns = chosen_ns + [ns] + [CANDIDATES[b][0][0] for b in BUCKETS[k + 1:]]
            tnw = chosen_nw + [nw] + [CANDIDATES[b][0][1] for b in BUCKETS[k + 1:]]
            t = _time_batch(Hs, (BUCKETS, tns, tnw))
            res.append((t, ns, nw))
            if verbose:
                print(f"bucket <= {bmax}: ns={ns} nw={nw}: {t:.3f} s")
        res.sort()
        timings[str(bmax)] = [[ns, nw, t] for t, ns, nw in res]
        chosen_ns.append(res[0][1])
        chosen_nw.append(res[0][2])
    api.set_batched_table(BUCKETS, chosen_ns, chosen_nw)
    return {"max_n": BUCKETS, "ns": chosen_ns, "nw": chosen_nw, "timings": timings}


if __name__ == "__main__":
    print(json.dumps(autotune_batched(verbose=True)))


def autotune_batched_nmin(lo=32, hi=768, seed=11, count=None, verbose=False):
    """Tune the batched engine's double-shift crossover nmin (blocks of at
    most nmin rows are finished by double-shift QR) with the current table,
    on one mixed batch of sizes uniform in [lo, hi]; returns
    {"nmin": best, "timings": {nmin: seconds}}."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    count = count or 2 * sms
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=count)
    Hs = []
    for i, n in enumerate(sizes):
        H = inputs.hessrand(int(n), [seed, i])
        Hs.append(torch.from_numpy(np.ascontiguousarray(H.T)).cuda().t())
    timings = {}
    for nmin in NMIN_CANDIDATES:
        Ss = [h.clone() for h in Hs]
        Zs = [api.new_colmajor(h.shape[0]) for h in Hs]
        wrs = [torch.empty(h.shape[0], dtype=torch.float64, device="cuda") for h in Hs]
        wis = [torch.empty_like(w) for w in wrs]
        api.schur_batched_inplace(Ss, Zs, wrs, wis, nmin=nmin)      # capture
        for s_, h in zip(Ss, Hs):
            s_.copy_(h)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = api.schur_batched_inplace(Ss, Zs, wrs, wis, nmin=nmin)
        e1.record()
        torch.cuda.synchronize()
        timings[nmin] = float("inf") if any(info) else e0.elapsed_time(e1) / 1e3
        if verbose:
            print(f"nmin={nmin}: {timings[nmin]:.3f} s")
    best = min(timings, key=timings.get)
    return {"nmin": best, "timings": timings}


SINGLE_CANDIDATES = {
    "n_shifts": [64, 96, 128],
    "aed_window": [96, 128, 160],
    "bulges_per_chain": [8, 12, 16],
}


def autotune_single(n=4096, seed=2021, candidates=None, verbose=False):
    """Tune the single-matrix path's shifts per sweep, AED window and bulges
    per chase chain (the chase window follows: 6 x bulges, at most 112) on
    one hess_n matrix of order n: a coordinate search over the candidate
    lists, each setting timed with CUDA events after a warm-up run.  Returns
    {"best": {...}, "seconds": t, "timings": [(settings, seconds), ...]}."""
    cand = candidates or SINGLE_CANDIDATES
    H = inputs.hessrand(n, seed)
    H0 = torch.from_numpy(np.ascontiguousarray(H.T)).cuda().t()
    S = api.new_colmajor(n)
    Z = api.new_colmajor(n)
    wr = torch.empty(n, dtype=torch.float64, device="cuda")
    wi = torch.empty_like(wr)
    stream = torch.cuda.current_stream()

    def run(cfg):
        o = api._lib.make_opts(stream.cuda_stream, **cfg)
        S.copy_(H0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc = api.schur_inplace(S, Z, wr, wi, o)
        e1.record()
        torch.cuda.synchronize()
        return float("inf") if rc else e0.elapsed_time(e1) / 1e3

    best = {k: v[len(v) // 2] for k, v in cand.items()}
    run(best)
    best_t = run(best)
    log = [(dict(best), best_t)]
    for key, values in cand.items():
        for v in values:
            if v == best[key]:
                continue
            cfg = dict(best, **{key: v})
            t = run(cfg)
            log.append((cfg, t))
            if verbose:
                print(cfg, f"{t:.3f} s")
            if t < best_t:
                best, best_t = cfg, t
    return {"best": best, "seconds": best_t, "timings": log}
