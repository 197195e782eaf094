"""The benchmark's reference arm (the oracle timed on the host cores): one
JSON line with the contract's keys, alone and under a two-rank launch
(rank 0 alone runs and prints; the other rank exits cleanly)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--steps", "1", "--warmup", "1", "--ref-budget", "0.3"]


def _lines(out: str):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check(line):
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "e2e",
              "cpu_baseline", "config"):
        assert k in line, k
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0])


def test_reference_arm_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2", *ARGS]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0])
    assert lines[0]["n_gpus"] == 2


def test_reference_config_matches_the_gpu_arm():
    """Both arms describe the workload with the same dict."""
    sys.path.insert(0, ROOT)
    import bench
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True, timeout=600)
    line = _lines(r.stdout)[0]
    assert line["config"] == bench.workload_config("seven", 1, "f32")


def test_cpu_baseline_all_cores_leg():
    """The oracle on several spawned processes at once: every process plans
    and simulates its own collective; the bytes add up and the line states
    the process count."""
    sys.path.insert(0, ROOT)
    import bench
    b, t, desc = bench.oracle_all_cores(0.3, 2)
    assert b > 0 and 0.3 <= t < 5.0 and "2 processes" in desc
    b1, t1 = bench._simulate_for("scatter", 0.2)
    assert b1 > 0 and t1 >= 0.2
