"""Benchmark: FP64 Hessenberg -> real Schur reduction (multishift QR + AED) on GB300.

Workload (default): one n = 20000 Hessenberg matrix of the paper's hess_n family
(Sec. 5.3: N(0,1) on and above the diagonal, chi(n-i) subdiagonal), seed 2023,
Z accumulated from the identity.  A step is one full reduction S = Z^T H Z
with the input already resident in HBM (a device copy restores H before each
step).  The matrix (3.2 GB each for H and Z) is larger than L2, so no flush
is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  metric/unit: seconds per n = 20000 reduction (lower is
better).  With N GPUs every rank reduces its own matrix (replicas; the
method has no data-parallel exchange at this size), value = max-over-ranks
time / N.  `roofline` refers to the dominant kernel, the off-window product
(k_apply_u), timed by CUDA events on its launch stream inside the library.
`cpu_baseline` times the CPU oracle (numpy, one thread) on a bounded sample and
scales it cubically to n = 20000.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.070e9 / 1e12   # TFLOP/s: SMs x FP64 FMA/clk x 2 x max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--ns", type=int, default=128)
    ap.add_argument("--nw", type=int, default=160)
    ap.add_argument("--seed", type=int, default=2023)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched (4096 x n in [32,768]) and backward (256 x n in [64,1024]) metrics")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi, 200 ms) during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# order of the CPU oracle sample: ~10 s of one-thread work on the hosts used
CPU_SAMPLE_N = 400


def cpu_baseline_sample(n_sample=CPU_SAMPLE_N, seed=2023):
    """Time the CPU oracle (one thread) on a bounded sample: one hess_n
    reduction of order n_sample, with the same shift/window rules."""
    code = (
        "import os, sys, time, json\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from oracle import qr\n"
        "from paper_2007_03576_gb300 import inputs\n"
        f"H = inputs.hessrand({n_sample}, {seed})\n"
        "t = time.perf_counter()\n"
        "S, Z, wr, wi, info = qr.schur(H)\n"
        "print(json.dumps({'sec': time.perf_counter() - t, 'info': info}))\n"
    )
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])["sec"]


L2_BYTES = 129e6    # GB300 L2


def needs_flush(n):
    """Whether a step's matrices fit in L2 (then L2 is flushed before each step)."""
    return 8.0 * n * n < 2 * L2_BYTES


def bench_config(args, world=1):
    """The workload description shared by both arms of the bench."""
    n = args.n
    mb = 8.0 * n * n / 1e6
    size = f"{mb / 1e3:.1f} GB" if mb >= 1e3 else f"{mb:.0f} MB"
    l2 = (f"inputs smaller than 2x L2 ({size} per matrix): L2 flushed before each step by a 512 MB write"
          if needs_flush(n) else f"inputs larger than L2 ({size} per matrix), no flush")
    return {"workload": f"hess_n n={n} (Sec. 5.3) Hessenberg -> real Schur, Z accumulated, seed {args.seed}",
            "n": n, "n_shifts": args.ns, "aed_window": args.nw, "deflation": "lapack-style",
            "l2": l2, "parallelism": f"replicas x{world}"}


def reference_arm(args):
    """--impl reference: the CPU oracle as it stands, each step one bounded
    sample (one hess_n reduction of order CPU_SAMPLE_N), scaled cubically to n."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_sample = CPU_SAMPLE_N
    for _ in range(args.warmup):
        cpu_baseline_sample(n_sample, args.seed)
    secs = [cpu_baseline_sample(n_sample, args.seed) for _ in range(args.steps)]
    t = sum(secs) / len(secs)
    scale = (args.n / n_sample) ** 3
    value = t * scale
    sample = (f"oracle (numpy FP64, 1 thread) reduction of one n={n_sample} hess_n matrix per step, "
              f"{t:.2f} s, scaled by (n/{n_sample})^3 to n={args.n}")
    line = {
        "impl": "reference", "metric": f"n={args.n} FP64 Schur time", "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, args.gpus),
        "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def secondary_metrics(api, inputs, torch, np):
    """The other two metrics of the workload list, each next to the plain
    single-matrix path on the same GPU:
      batched:  4096 hess_n matrices, n uniform in [32, 768] (seed 2024), one
                persistent graph-captured launch -> matrices/s;
      backward: 256 hess_n matrices, n uniform in [64, 1024] (seed 2025), loss
                sum |lambda|^2 -> batched backward time / batched forward time."""

    def load(sizes, seed):
        Hs = []
        for b, n in enumerate(sizes):
            H = inputs.hessrand(int(n), [seed, b])
            Hs.append(torch.from_numpy(np.ascontiguousarray(H.T)).cuda().t())
        return Hs

    def buffers(Hs):
        Ss = [h.clone() for h in Hs]
        Zs = [api.new_colmajor(h.shape[0]) for h in Hs]
        wr = [torch.empty(h.shape[0], dtype=torch.float64, device="cuda") for h in Hs]
        wi = [torch.empty_like(w) for w in wr]
        return Ss, Zs, wr, wi

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    out = {}
    sizes = inputs.batch_sizes(4096, 32, 768, 2024)
    Hs = load(sizes, 2024)
    bufs = buffers(Hs)
    api.schur_batched_inplace(*bufs)                     # warm-up
    for s_, h in zip(bufs[0], Hs):
        s_.copy_(h)
    t, info = timed(lambda: api.schur_batched_inplace(*bufs))
    single = []
    for h in Hs[:16]:
        S1, Z1 = h.clone(), api.new_colmajor(h.shape[0])
        w1 = torch.empty(h.shape[0], dtype=torch.float64, device="cuda")
        w2 = torch.empty_like(w1)
        o = api._lib.make_opts(torch.cuda.current_stream().cuda_stream)
        ts, _ = timed(lambda: api.schur_inplace(S1, Z1, w1, w2, o))
        single.append(ts)
    out["batched"] = {"workload": "4096 hess_n, n uniform in [32,768], seed 2024", "mats_per_s": 4096 / t,
                      "seconds": t, "failed": int(sum(1 for i in info if i)), "launches": 2,
                      "single_path_mats_per_s": len(single) / sum(single),
                      "single_path_sample": "first 16 matrices of the batch, one schur_hessenberg call each"}
    del Hs, bufs
    torch.cuda.empty_cache()
    sizes = inputs.batch_sizes(256, 64, 1024, 2025)
    Hs = load(sizes, 2025)
    bufs = buffers(Hs)
    api.schur_batched_inplace(*bufs)                     # warm-up
    for s_, h in zip(bufs[0], Hs):
        s_.copy_(h)
    tf, info = timed(lambda: api.schur_batched_inplace(*bufs))
    Ss, Zs, wr, wi = bufs
    gr = [2 * a for a in wr]
    gi = [2 * b for b in wi]
    api.eig_backward_batched(Ss, Zs, wr, wi, gr, gi)     # warm-up
    tb, _ = timed(lambda: api.eig_backward_batched(Ss, Zs, wr, wi, gr, gi))
    one_f, one_b = 0.0, 0.0
    for h in Hs[:8]:
        ts, (S1, Z1, a, b, rc) = timed(lambda: api.schur(h))
        tg, _ = timed(lambda: api.eig_backward(S1, Z1, a, b, 2 * a, 2 * b))
        one_f += ts
        one_b += tg
    out["backward"] = {"workload": "256 hess_n, n uniform in [64,1024], seed 2025, L = sum |lambda|^2",
                       "forward_s": tf, "backward_s": tb, "backward_over_forward": tb / tf,
                       "failed": int(sum(1 for i in info if i)),
                       "single_path_backward_over_forward": one_b / one_f,
                       "single_path_sample": "first 8 matrices, schur_hessenberg + schur_eig_backward each"}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2007_03576_gb300 import api, inputs, _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.n
    # input: hess_n, generated on the host once, resident in HBM
    Ht = inputs.hessrand_colmajor(n, args.seed + rank)
    H0 = torch.from_numpy(Ht).cuda().t()          # column-major view, ld = n
    H = api.new_colmajor(n)
    Z = api.new_colmajor(n)
    wr = torch.empty(n, dtype=torch.float64, device="cuda")
    wi = torch.empty(n, dtype=torch.float64, device="cuda")
    ws_bytes = api.workspace_bytes(n, n_shifts=args.ns, aed_window=args.nw)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def opts(timing):
        o = _lib.make_opts(stream.cuda_stream, n_shifts=args.ns, aed_window=args.nw, timing=timing)
        o.workspace = ws.data_ptr()
        o.workspace_bytes = ws_bytes
        return o

    o_plain = opts(0)
    o_timed = opts(1)

    flush = torch.empty(64 * 2 ** 20, dtype=torch.float64, device="cuda") if needs_flush(n) else None

    def step(o):
        if flush is not None:
            flush.fill_(1.0)
        H.copy_(H0)
        rc = api.schur_inplace(H, Z, wr, wi, o)
        if rc != 0:
            raise RuntimeError(f"schur_hessenberg returned {rc}: {_lib.status(rc)}")

    for _ in range(args.warmup):
        step(o_plain)
    torch.cuda.synchronize()

    # timed region: K steps, CUDA events on the launching stream; the library
    # records per-phase CUDA events (timing=1) for the roofline of k_apply_u
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        step(o_timed)
        stats.append(api.last_stats())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    t_step = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t_step, op=dist.ReduceOp.MAX)
    ms = float(t_step.item())

    # correctness probe of the last step (cheap, O(n^2)): trace invariant,
    # residual and orthogonality along a random vector
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    resid = float(((Z @ (H @ (Z.t() @ x))) - H0 @ x).norm() / (torch.linalg.matrix_norm(H0) * x.norm()))
    orth = float((Z.t() @ (Z @ x) - x).norm() / x.norm())
    trace_err = abs(float(wr.sum()) - float(torch.diagonal(H0).sum())) / float(torch.diagonal(H0).abs().sum())

    # end to end: pinned host input, host->device copy, reduction, device->host
    # copy of the result (S, Z, eigenvalues), all inside the timed region
    e2e = None
    if not args.no_e2e:
        Hh = torch.from_numpy(Ht).pin_memory()      # H^T row-major == H column-major
        Sh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        Zh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        wh = torch.empty((2, n), dtype=torch.float64).pin_memory()
        Hd = H.t()                                    # row-major storage of the column-major buffer
        Zd = Z.t()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Hd.copy_(Hh, non_blocking=True)
        rc = api.schur_inplace(H, Z, wr, wi, o_plain)
        if rc != 0:
            raise RuntimeError(f"schur_hessenberg returned {rc}")
        Sh.copy_(Hd, non_blocking=True)
        Zh.copy_(Zd, non_blocking=True)
        wh[0].copy_(wr, non_blocking=True)
        wh[1].copy_(wi, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = {"value": float(t.item()) / world, "unit": "s", "h2d_bytes_per_step": n * n * 8,
               "d2h_bytes_per_step": 2 * n * n * 8 + 2 * n * 8, "steps": 1}

    # in-run FP64 GEMM reference (cuBLAS DGEMM through torch, a library run
    # used only as a denominator)
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    a @ b
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record()
    for _ in range(3):
        a @ b
    g1.record()
    torch.cuda.synchronize()
    dgemm_tflops = 3 * 2 * 8192 ** 3 / (g0.elapsed_time(g1) / 1e3) / 1e12
    del a, b

    sec = None if args.no_secondary else secondary_metrics(api, inputs, torch, np)

    st = stats[-1]
    upd_flops = sum(s["sweep_gemm_flops"] for s in stats)
    # kernel time of the sweep products on all three streams (H rows on the
    # main stream, H rows above the windows on the side stream, Z on the
    # low-priority stream); they overlap in wall time, so this is the sum of
    # the products' own durations
    upd_ms = sum(s["t_update_ms"] + s["t_z_ms"] for s in stats)
    upd_launches = sum(s["update_launches"] for s in stats)
    achieved = upd_flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else None
    launches = int(sum(s["kernel_launches"] for s in stats) / len(stats))

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        n_sample = CPU_SAMPLE_N
        t = cpu_baseline_sample(n_sample, args.seed)
        cpu = {"value": t * (n / n_sample) ** 3, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"oracle (numpy FP64, 1 thread) on one n={n_sample} hess_n reduction: {t:.2f} s, "
                         f"scaled by (n/{n_sample})^3"}
    phase_ms = {k: round(st[k], 1)
                for k in ("t_chase_ms", "t_update_ms", "t_z_ms", "t_aed_ms", "t_aed_update_ms", "t_small_ms")}
    line = {
        "metric": f"n={n} FP64 Schur time",
        "value": ms / 1e3 / world,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(args, world),
        "roofline": {"bound": "alu", "kernel": "k_apply_u (off-window products, FP64 FFMA)",
                     "achieved": achieved, "peak": FP64_PEAK_DERIVED, "unit": "TFLOP/s",
                     "frac": (achieved / FP64_PEAK_DERIVED) if achieved else None, "traffic": None,
                     "peak_note": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                     "dgemm_tflops_same_run": dgemm_tflops,
                     "frac_of_dgemm": (achieved / dgemm_tflops) if achieved else None,
                     "launches": upd_launches, "flops": upd_flops, "ms": upd_ms},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
        "phase_ms": phase_ms,
        "iterations": {"aed": st["aed_steps"], "sweeps": st["sweeps"], "deflated_by_aed": st["deflated_by_aed"]},
        "flops": {"reflector_algorithmic": st["reflector_flops"], "sweep_gemm_executed": st["sweep_gemm_flops"],
                  "aed_gemm_executed": st["aed_gemm_flops"]},
        "secondary": sec,
        "check": {"residual_probe": resid, "orthogonality_probe": orth, "trace_rel_err": trace_err},
        "context": "paper Table 4: syn_20000 StarNEig 68 s on 25 Skylake cores (different matrix family)",
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
