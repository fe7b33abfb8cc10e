#!/usr/bin/env python
"""Throughput benchmark of the partitioned skyline hot path on the GPU.

Workload: 1,000,000 anticorrelated FP32 points, d = 6 (seeded synthetic
data; the paper's own generator is unstated).  One step runs four exact
skyline queries over the device-resident input, the partitioned method
with Sliced (p = 64) and Angular (m = 4,2,2,2,2 -> p = 64) partitioning,
each without and with Sorted representatives (1 per partition), every local
skyline of a query in one persistent cooperative launch and the sequential
final merge.  The metric is input points per second at the exact result
(4 x N points per step).  The same step with one launch per partition is
reported as `plain`; `e2e` runs it through the C ABI from host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
Under torchrun every rank runs the same workload on its own GPU (replicas;
the path has no data exchange between GPUs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "skyline input points/sec at exact result, batched vs plain GPU; p99 latency"
N, D, SEED = 1_000_000, 6, 1
VARIANTS = [
    ("sliced", dict(scheme="sliced", p=64)),
    ("sliced_rep", dict(scheme="sliced", p=64, rep="sorted")),
    ("angular", dict(scheme="angular", slices=[4, 2, 2, 2, 2])),
    ("angular_rep", dict(scheme="angular", slices=[4, 2, 2, 2, 2], rep="sorted")),
]
WORKLOAD = (f"anticorrelated FP32 N={N} d={D} seed={SEED}; Sliced p=64 and Angular (4,2,2,2,2), "
            "each without and with 1 Sorted representative per partition; sequential merge")
L2_FLUSH_BYTES = 256 << 20
SM_COUNT = 152


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_workcounts():
    p = os.path.join(ROOT, "tests", "golden", "workcounts_ant_1m_d6.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        return json.load(fh)["variants"]


def cpu_oracle_sample(n_sample: int):
    """Times the CPU oracle (single-threaded C, as it stands) on the same
    variants over the first n_sample points of the same generator."""
    from oracle import oracle as O
    from paper_2411_14968_gb300 import datagen
    x = datagen.anticorrelated(n_sample, D, SEED)
    kw = {
        "sliced": dict(scheme=O.SLICED, p=64),
        "sliced_rep": dict(scheme=O.SLICED, p=64, rep=O.REP_SORTED),
        "angular": dict(scheme=O.ANGULAR, slices=[4, 2, 2, 2, 2]),
        "angular_rep": dict(scheme=O.ANGULAR, slices=[4, 2, 2, 2, 2], rep=O.REP_SORTED),
    }
    O.build()
    t = time.perf_counter()
    for name, _ in VARIANTS:
        O.partitioned(x, **kw[name])
    return time.perf_counter() - t, len(VARIANTS) * n_sample


def reference_arm(args, rank, world):
    """The CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    n_sample = 25_000
    for _ in range(args.warmup):
        cpu_oracle_sample(n_sample)
    secs, pts = 0.0, 0
    for _ in range(args.steps):
        s, p = cpu_oracle_sample(n_sample)
        secs += s
        pts += p
    value = pts / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_points": n_sample},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n_sample} points of the same generator, 4 variants per step"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gpu_arm(args, rank, world, local):
    import torch
    from paper_2411_14968_gb300 import datagen, native

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        if world == 1:
            return v
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    x = datagen.anticorrelated(N, D, SEED)
    xt = torch.from_numpy(x).to(dev)
    ctx = native.Context(local)
    ctx.set_timing(True)
    persistent = {name: native.make_params(exec="persistent", **kw) for name, kw in VARIANTS}
    plain = {name: native.make_params(exec="plain", **kw) for name, kw in VARIANTS}
    out = torch.empty(N, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(pmap, acc=None):
        counts = {}
        for name, p in pmap.items():
            idx = ctx.skyline(xt, params=p, out=out)
            st = ctx.stats()
            counts[name] = int(idx.shape[0])
            if acc is not None:
                acc["launches"] += st["launches"]
                acc["dom_ms"] += st["ms_dom_local"] + st["ms_dom_merge"]
                acc["per_variant"].setdefault(name, []).append(st)
        return counts

    def timed(pmap, k):
        acc = {"launches": 0, "dom_ms": 0.0, "per_variant": {}}
        ms = []
        barrier()
        torch.cuda.synchronize()
        for _ in range(k):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(pmap, acc)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier()
        return ms, acc

    # warm-up (also checks that every variant gives the same set: Prop. 1)
    ref_counts = None
    for _ in range(max(args.warmup, 3)):
        c1 = step(persistent)
        c2 = step(plain)
        if ref_counts is None:
            ref_counts = c1
        assert len(set(c1.values()) | set(c2.values())) == 1, (c1, c2)

    clocks = ClockSampler(local)
    clocks.start()
    ms, acc = timed(persistent, args.steps)
    clk = clocks.stop()
    total_s = max_over_ranks(sum(ms) / 1e3)
    pts_per_step = N * len(VARIANTS)
    value = pts_per_step * args.steps * world / total_s

    # plain form: one launch per partition
    ms_plain, acc_plain = timed(plain, max(1, args.steps))
    plain_s = max_over_ranks(sum(ms_plain) / 1e3)
    plain_value = pts_per_step * len(ms_plain) * world / plain_s

    # end to end through the C ABI from pinned host buffers
    xh = torch.from_numpy(x).pin_memory().numpy()
    sky_total = sum(ref_counts.values())
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k_e2e = max(1, args.steps)
    for _ in range(k_e2e):
        for name, p in persistent.items():
            ctx.skyline(xh, params=p)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = pts_per_step * k_e2e * world / e2e_s

    # roofline of the dominance kernel (k_engine): algorithmic compares
    # (oracle test count x d) over its measured launch time
    wc = load_workcounts()
    roof = None
    dom_ms_per_step = acc["dom_ms"] / args.steps
    if wc:
        tests = sum(wc[name]["local_tests"] + wc[name]["merge_tests"] for name, _ in VARIANTS)
        achieved = tests * D / (dom_ms_per_step * 1e-3) / 1e12
        peak = args.compare_peak_tcmp
        roof = {"bound": "alu", "kernel": "k_engine (dominance tiles, local + merge launches)",
                "achieved": achieved, "peak": peak, "unit": "Tcmp/s", "frac": achieved / peak,
                "traffic": None, "algorithmic_tests_per_step": tests,
                "kernel_ms_per_step": dom_ms_per_step,
                "kernel_share_of_step": dom_ms_per_step / (sum(ms) / len(ms))}

    # per-variant breakdown (medians over the timed steps)
    per_variant = {}
    for name, sts in acc["per_variant"].items():
        per_variant[name] = {
            "skyline": ref_counts[name],
            "local_union": sts[-1]["local_union"],
            "rounds_local": sts[-1]["rounds_local"],
            "rounds_merge": sts[-1]["rounds_merge"],
            "ms_total": statistics.median(s["ms_total"] for s in sts),
            "ms_dom_local": statistics.median(s["ms_dom_local"] for s in sts),
            "ms_dom_merge": statistics.median(s["ms_dom_merge"] for s in sts),
            "ms_phase": [round(statistics.median(s["ms_phase"][i] for s in sts), 4) for i in range(6)],
        }

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_sample = 100_000
        secs, pts = cpu_oracle_sample(n_sample)
        cpu = {"value": pts / secs, "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n_sample} points of the same generator, the 4 variants once ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded anticorrelated generator; the paper's generator is unstated)",
            "config": {"workload": WORKLOAD, "points_per_step": pts_per_step, "exec": "persistent",
                       "l2": "flushed between timed steps (256 MB write outside the timed events)",
                       "parallelism": f"replicas x{world}"},
            "plain": {"value": plain_value, "unit": "points/s", "ms_per_step": sum(ms_plain) / len(ms_plain),
                      "speedup_persistent_over_plain": value / plain_value},
            "e2e": {"value": e2e_value, "unit": "points/s",
                    "h2d_bytes_per_step": len(VARIANTS) * N * D * 4,
                    "d2h_bytes_per_step": 4 * sky_total + len(VARIANTS) * 128},
            "gpu_launches": int(acc["launches"]),
            "clocks": clk,
            "roofline": roof,
            "cpu_baseline": cpu,
            "variants": per_variant,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # FP32 compare peak: 152 SMs x 64 compare lanes per SM per clock x 2.07 GHz
    # (the compare-rate probe of the library measures 58.6 per SM per clock)
    ap.add_argument("--compare-peak-tcmp", type=float, default=SM_COUNT * 64 * 2.07e9 / 1e12)
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    gpu_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
