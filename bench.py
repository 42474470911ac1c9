"""Benchmark: FP64 Hessenberg -> real Schur reduction (multishift QR + AED) on GB300.

Workload (default): one n = 20000 Hessenberg matrix of the paper's hess_n family
(Sec. 5.3: N(0,1) on and above the diagonal, chi(n-i) subdiagonal), seed 2023,
Z accumulated from the identity, 160 shifts, AED window 160, AED repeated
above 20 % deflation (tuned settings).  A step is one full reduction S = Z^T H Z
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
import ctypes
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--ns", type=int, default=160)
    ap.add_argument("--nw", type=int, default=160)
    ap.add_argument("--seed", type=int, default=2023)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched (4096 x n in [32,768]) and backward (256 x n in [64,1024]) metrics")
    ap.add_argument("--no-checks", action="store_true", help="skip the full-size checks of the last reduction")
    ap.add_argument("--no-cpu-lapack", action="store_true", help="skip the LAPACK (scipy.linalg.schur) CPU sample")
    ap.add_argument("--nibble", type=int, default=20,
                    help="repeat AED when it deflates more than this percent of the window (tuned at n = 20000: "
                         "14 / 20 / 25 / 30 gave 41.0 / 40.3 / 40.7 / 41.6 s; 0 = the library default, 14)")
    ap.add_argument("--split-products", action="store_true",
                    help="opts.split_products = 1: a chase step's far left products beside the next chase step")
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
            "n": n, "n_shifts": args.ns, "aed_window": args.nw, "nibble": getattr(args, "nibble", 0) or 14,
            "deflation": "lapack-style",
            "l2": l2, "parallelism": f"replicas x{world}",
            "products": "split over four streams" if getattr(args, "split_products", False) else "three streams"}


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


def secondary_metrics(api, inputs, torch, np, peak=None):
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
    bst = api.last_stats()
    single = []
    for h in Hs[:16]:
        S1, Z1 = h.clone(), api.new_colmajor(h.shape[0])
        w1 = torch.empty(h.shape[0], dtype=torch.float64, device="cuda")
        w2 = torch.empty_like(w1)
        o = api._lib.make_opts(torch.cuda.current_stream().cuda_stream)
        ts, _ = timed(lambda: api.schur_inplace(S1, Z1, w1, w2, o))
        single.append(ts)
    bfl = bst["reflector_flops"]
    out["batched"] = {"workload": "4096 hess_n, n uniform in [32,768], seed 2024", "mats_per_s": 4096 / t,
                      "seconds": t, "failed": int(sum(1 for i in info if i)), "launches": 2,
                      "graph_replayed": bst["graph_built"] == 0,
                      "algorithmic_flops": bfl, "algorithmic_tflops": bfl / t / 1e12,
                      "frac_of_peak": (bfl / t / 1e12 / peak) if peak else None,
                      "flops_note": "counted by the kernel: 4 nr flops per row/column entry of each reflector "
                                    "of order nr it applies, 2 nw^2 per vector of each AED window product",
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
    del Hs, bufs
    torch.cuda.empty_cache()
    # the phases around the iteration at n = 4096: Householder reduction of a
    # dense N(0,1) matrix (H and Q), eigenvectors of a hess_n Schur form
    n = 4096
    A = inputs.gaussian(n, 2022)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    api.hessenberg_reduce(Ad)                           # warm-up
    tr, _ = timed(lambda: api.hessenberg_reduce(Ad))
    rfl = api.last_stats()["flops"]
    H = inputs.hessrand(n, 2021)
    Hd = torch.from_numpy(np.ascontiguousarray(H.T)).cuda().t()
    tf4, (S, Z, wr1, wi1, _) = timed(lambda: api.schur(Hd))
    api.eigenvectors(S, Z, wr1, wi1)                    # warm-up
    te, _ = timed(lambda: api.eigenvectors(S, Z, wr1, wi1))
    efl = api.last_stats()["flops"]
    api.eig_backward(S, Z, wr1, wi1, 2 * wr1, -2 * wi1)  # warm-up
    tb4, _ = timed(lambda: api.eig_backward(S, Z, wr1, wi1, 2 * wr1, -2 * wi1))
    bfl = api.last_stats()["flops"]
    out["phases_n4096"] = {
        "reduction": {"workload": "dense N(0,1) n=4096 seed 2022 -> H, Q", "seconds": tr,
                      "algorithmic_flops": rfl, "tflops": rfl / tr / 1e12,
                      "frac_of_peak": (rfl / tr / 1e12 / peak) if peak else None},
        "eigenvectors": {"workload": "hess_n n=4096 seed 2021 Schur form -> X = Z X_S", "seconds": te,
                         "algorithmic_flops": efl, "tflops": efl / te / 1e12,
                         "frac_of_peak": (efl / te / 1e12 / peak) if peak else None},
        "backward": {"workload": "hess_n n=4096 seed 2021, L = sum Re lambda^2 -> dL/dH (blocked vector path)",
                     "seconds": tb4, "forward_s": tf4, "backward_over_forward": tb4 / tf4,
                     "algorithmic_flops": bfl, "tflops": bfl / tb4 / 1e12,
                     "frac_of_peak": (bfl / tb4 / 1e12 / peak) if peak else None},
        "flops_note": "reduction (10/3 + 4/3) n^3, eigenvectors n^3/3 + n^3 (the counts of the same work in LAPACK); "
                      "backward: the GEMM flops it issues (two n^3/3 substitutions, about n^3/3 + n^3 + 2 n^3 "
                      "for Z Re(sum e w x^T) Z^T)"}
    return out


# DRAM traffic of k_apply_u from one ncu capture (profiles/ncu_apply_u_n5000.md:
# dram__bytes_read.sum + dram__bytes_write.sum over the captured launches,
# divided by the flops those launches execute), valid for the kernel source
# whose hash is recorded; scaled to an average launch of the benchmark by its
# executed flops.
APPLY_U_CAPTURE = {"sha": "9fd69261561f1af4", "dram_bytes_per_exec_flop": 7.8669e6 / (1739896 * 64),
                   "case": "n=5000 hess_n, 64 shifts, window 128; 3 launches of k_apply_u<64> after 300"}


def apply_u_source_hash():
    """Hash of k_apply_u's source (the part of kernels.cu from the product
    kernel's comment to its launcher)."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2007_03576_gb300", "csrc", "kernels.cu")).read()
    a = src.find("// Off-window products (Sec. 3.2.1 left/right update)")
    b = src.find("cudaError_t launch_apply_u(")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16] if a >= 0 and b > a else None


def apply_u_traffic(exec_flops_per_launch):
    """DRAM bytes of an average k_apply_u launch, from the capture above; None
    when there is no capture of the current kernel source."""
    cap = APPLY_U_CAPTURE
    if not cap or not exec_flops_per_launch or cap["sha"] != apply_u_source_hash():
        return None
    return cap["dram_bytes_per_exec_flop"] * exec_flops_per_launch


def host_cpu():
    """CPU model and the number of host cores (for the CPU baselines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def lapack_schur_sample():
    """LAPACK's real Schur factorisation (scipy.linalg.schur = dgees, OpenBLAS
    on all host cores) of the n = 256 and n = 4096 hess_n workloads: a tuned
    CPU library beside the plain oracle (not the method's code path)."""
    code = (
        "import sys, time, json\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import scipy, scipy.linalg\n"
        "from paper_2007_03576_gb300 import inputs\n"
        "out = {}\n"
        "for n, seed in ((256, 2020), (4096, 2021)):\n"
        "    H = inputs.hessrand(n, seed)\n"
        "    t = time.perf_counter()\n"
        "    scipy.linalg.schur(H, overwrite_a=True, check_finite=False)\n"
        "    out[str(n)] = time.perf_counter() - t\n"
        "out['scipy'] = scipy.__version__\n"
        "print(json.dumps(out))\n"
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def fp64_peaks(api, _lib, torch, local):
    """In-run FP64 rates: the library's FMA throughput probe (the products'
    instruction; the roofline denominator) with clocks sampled while it runs,
    and cuBLAS DGEMM 8192^3 (a library run, for reference)."""
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    blocks = 8 * nsm
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    o = _lib.make_opts(stream.cuda_stream)
    flops = ctypes.c_double()
    lib = _lib.load()

    def probe(iters):
        assert lib.schur_fp64_fma_probe(iters, blocks, out.data_ptr(), ctypes.byref(flops), ctypes.byref(o)) == 0
        return flops.value

    probe(2000)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    rates = []
    for _ in range(8):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = probe(60000)
        e1.record(stream)
        torch.cuda.synchronize()
        rates.append(f / (e0.elapsed_time(e1) / 1e3) / 1e12)
    clocks = sampler.stop()
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    a @ b
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record()
    for _ in range(3):
        a @ b
    g1.record()
    torch.cuda.synchronize()
    dgemm = 3 * 2 * 8192 ** 3 / (g0.elapsed_time(g1) / 1e3) / 1e12
    del a, b
    return {"fma_probe_tflops": max(rates), "fma_probe_median_tflops": statistics.median(rates),
            "fma_probe_clocks": clocks, "dgemm_tflops": dgemm,
            "fma_probe": f"{blocks} blocks x 256 threads x 8 FMA chains, best of 8 launches, CUDA events"}


def full_checks(torch, np, H0, S, Z, wr, wi, n, seed):
    """Checks of the last reduction at full size (after the timed region):
    backward error ||H Z - Z S||_F / ||H||_F and ||Z^T Z - I||_F / sqrt(n)
    (Sec. 5.4) with cuBLAS products, the standardised quasi-triangular
    structure of S and its agreement with wr/wi, and, when a stored LAPACK
    spectrum of this matrix exists, a one-to-one nearest matching of the
    eigenvalues to it."""
    out = {}
    nh = float(torch.linalg.matrix_norm(H0))
    R = H0 @ Z
    R -= Z @ S
    out["residual_fro"] = float(torch.linalg.matrix_norm(R)) / nh
    del R
    G = Z.t() @ Z
    G.diagonal().sub_(1.0)
    out["orthogonality_fro_over_sqrt_n"] = float(torch.linalg.matrix_norm(G)) / math.sqrt(n)
    del G
    torch.cuda.empty_cache()
    below = float(torch.tril(S, -2).abs().max()) if n > 2 else 0.0
    sub = torch.diagonal(S, -1)
    nz = sub != 0
    adjacent = int((nz[1:] & nz[:-1]).sum()) if n > 2 else 0
    d = torch.diagonal(S)
    sup = torch.diagonal(S, 1)
    j = torch.nonzero(nz).flatten()
    eqdiag = int((d[j] != d[j + 1]).sum())
    sign = int((sup[j] * sub[j] >= 0).sum())
    wi_bad = int(((wi[j] <= 0) | (wi[j + 1] >= 0)).sum())
    out["structure_errors"] = {"below_subdiagonal_max": below, "adjacent_subdiagonals": adjacent,
                               "unequal_block_diagonal": eqdiag, "block_offdiag_sign": sign,
                               "wi_pairing": wi_bad, "blocks_2x2": int(j.numel())}
    out["structure_ok"] = below == 0.0 and adjacent == 0 and eqdiag == 0 and sign == 0 and wi_bad == 0
    path = os.path.join(ROOT, "tests", "golden", f"hess_n{n}_seed{seed}_eigvals.npy")
    if os.path.exists(path):
        from scipy.spatial import cKDTree
        ref = np.load(path)
        lam = wr.cpu().numpy() + 1j * wi.cpu().numpy()
        tree = cKDTree(np.stack([ref.real, ref.imag], axis=1))
        dist, idx = tree.query(np.stack([lam.real, lam.imag], axis=1))
        one_to_one = len(np.unique(idx)) == n
        hf = nh
        out["lapack_eigs"] = {"max_dist_over_normH": float(np.max(dist)) / hf,
                              "median_dist_over_normH": float(np.median(dist)) / hf,
                              "one_to_one": bool(one_to_one),
                              "within_1e-10_normH": int(np.sum(dist <= 1e-10 * hf)),
                              "reference": os.path.relpath(path, ROOT)}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2007_03576_gb300 import api, inputs, _lib, trace

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
        o = _lib.make_opts(stream.cuda_stream, n_shifts=args.ns, aed_window=args.nw, timing=timing,
                           split_products=1 if args.split_products else 0, nibble=args.nibble)
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

    # warm-up; the last warm-up step writes the timeline of its launches
    # (SCHUR_TRACE) for the union of the products' intervals
    trace_path = os.path.join(tempfile.gettempdir(), f"schur_bench_trace_{os.getpid()}.csv")
    for w in range(args.warmup):
        if w == args.warmup - 1:
            os.environ["SCHUR_TRACE"] = trace_path
        step(o_timed if w == args.warmup - 1 else o_plain)
        os.environ.pop("SCHUR_TRACE", None)
    torch.cuda.synchronize()
    traced_stats = api.last_stats()
    tsum = trace.summarize(trace_path) if os.path.exists(trace_path) else None
    if os.path.exists(trace_path):
        os.remove(trace_path)

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

    # checks of the last step at full size (outside the timed region)
    checks = None if args.no_checks else full_checks(torch, np, H0, H, Z, wr, wi, n, args.seed + rank)

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
        del Hh, Sh, Zh, wh

    del H0
    torch.cuda.empty_cache()
    peaks = fp64_peaks(api, _lib, torch, local)
    sec = None if args.no_secondary else secondary_metrics(api, inputs, torch, np,
                                                           max(peaks["fma_probe_tflops"], peaks["dgemm_tflops"]))

    st = stats[-1]
    # the dominant kernel, k_apply_u (the sweeps' off-window products on H's
    # rows, H's columns above the windows and Z): algorithmic flops = those
    # of applying the sweeps' 3x3 reflectors directly (12 per reflector and
    # row/column entry); executed flops = what the banded window products
    # compute; durations = the launches' CUDA-event times on their streams
    alg_flops = sum(s["reflector_flops"] for s in stats)
    exec_flops = sum(s["sweep_gemm_flops"] for s in stats)
    upd_ms = sum(s["t_update_ms"] + s["t_z_ms"] for s in stats)
    upd_launches = sum(s["update_launches"] for s in stats)
    achieved = alg_flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else None
    # the larger of the two in-run FP64 rates (the FMA probe, cuBLAS DGEMM)
    peak = max(peaks["fma_probe_tflops"], peaks["dgemm_tflops"])
    union_ms = tsum["union_ms"]["products"] if tsum else None
    achieved_union = (traced_stats["reflector_flops"] / (union_ms / 1e3) / 1e12) if union_ms else None
    launches = int(sum(s["kernel_launches"] for s in stats) / len(stats))
    traffic = apply_u_traffic(upd_launches and (exec_flops / upd_launches))

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        n_sample = CPU_SAMPLE_N
        t = cpu_baseline_sample(n_sample, args.seed)
        cpu = {"value": t * (n / n_sample) ** 3, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"oracle (numpy FP64, 1 thread) on one n={n_sample} hess_n reduction: {t:.2f} s, "
                         f"scaled by (n/{n_sample})^3", **host_cpu()}
        if not args.no_cpu_lapack:
            lap = lapack_schur_sample()
            cpu["lapack_schur_s"] = {k: v for k, v in lap.items() if k != "scipy"}
            cpu["lapack_note"] = (f"scipy {lap.get('scipy')} linalg.schur (LAPACK dgees via OpenBLAS, all "
                                  f"{os.cpu_count()} host cores) on hess_n n=256 (seed 2020) and n=4096 (seed 2021)")
            ref = os.path.join(ROOT, "tests", "golden", f"hess_n{n}_seed{args.seed}_eigvals.json")
            if os.path.exists(ref):
                cpu["lapack_offline"] = json.loads(open(ref).read())
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
        "roofline": {"bound": "alu", "kernel": "k_apply_u (off-window products of the sweeps, FP64 FMA)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_note": "measured in this run: max of the library's FP64 FMA probe "
                                  "(schur_fp64_fma_probe, clocks in peaks.fma_probe_clocks) and cuBLAS DGEMM 8192^3",
                     "achieved_note": "algorithmic flops (3x3 reflectors applied directly, 12 per entry) / "
                                      "sum of the launches' CUDA-event durations",
                     "achieved_union": achieved_union,
                     "frac_union": (achieved_union / peak) if achieved_union else None,
                     "union_note": "algorithmic flops / union of the products' intervals on the three streams "
                                   "(last warm-up step, SCHUR_TRACE)",
                     "executed_flops": exec_flops, "algorithmic_flops": alg_flops,
                     "executed_over_algorithmic": exec_flops / alg_flops if alg_flops else None,
                     "executed_tflops": exec_flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else None,
                     "launches": upd_launches, "ms": upd_ms, "union_ms": union_ms},
        "peaks": peaks,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
        "phase_ms": phase_ms,
        "timeline": ({k: round(v, 1) for k, v in tsum["union_ms"].items()} | {"span": round(tsum["span_ms"], 1)})
        if tsum else None,
        "iterations": {"aed": st["aed_steps"], "sweeps": st["sweeps"], "deflated_by_aed": st["deflated_by_aed"]},
        "flops": {"reflector_algorithmic": st["reflector_flops"], "sweep_gemm_executed": st["sweep_gemm_flops"],
                  "aed_gemm_executed": st["aed_gemm_flops"]},
        "secondary": sec,
        "check": checks,
        "context": "paper Table 4: syn_20000 StarNEig 68 s on 25 Skylake cores (different matrix family)",
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
