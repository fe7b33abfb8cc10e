"""The benchmark's reference arm (the CPU oracle, which needs no GPU) keeps
the JSON contract: one line with the metric, a positive value, its unit and
the CPU-baseline and end-to-end objects; under torchrun only rank 0 prints
and every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(out: str):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    ln = lines[0]
    assert ln["impl"] == "reference" and ln["metric"] == bench.METRIC
    assert ln["value"] > 0 and ln["unit"] == "points/s" and ln["higher_is_better"] is True
    assert ln["steps"] == 1 and ln["warmup"] == 0 and ln["n_gpus"] == 1
    cb = ln["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == ln["value"] and cb["sample"]
    e2e = ln["e2e"]
    assert e2e["value"] == ln["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert ln["config"]["workload"] == bench.WORKLOAD


def test_reference_arm_under_torchrun_prints_once():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
