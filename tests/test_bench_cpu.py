"""bench.py's reference arm on the CPU: one process, and two ranks under
torchrun (rank 0 alone runs the oracle and prints the line; the other rank
exits 0 without work).  The reference line carries the same metric, unit,
config and direction as the GPU arm's line."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _env():
    env = dict(os.environ)
    env.setdefault("OMP_NUM_THREADS", "1")
    return env


def _check_line(d, gpus):
    assert d["impl"] == "reference"
    assert d["metric"] == "n=20000 FP64 Schur time"
    assert d["unit"] == "s" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == gpus and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["n"] == 20000 and d["config"]["n_shifts"] == 160 and d["config"]["aed_window"] == 160 and d["config"]["nibble"] == 20
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=_env())
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


@pytest.mark.slow
def test_reference_arm_two_ranks_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=_env())
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 2)
