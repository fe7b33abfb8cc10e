#!/usr/bin/env python
"""Throughput benchmark of the partitioned skyline hot path on the GPU.

Workload: 1,000,000 anticorrelated FP32 points, d = 6 (seeded synthetic
data; the paper's own generator is unstated).  One step runs four exact
skyline queries over the device-resident input -- the partitioned method
with Sliced (p = 64) and Angular (m = 4,2,2,2,2 -> p = 64) partitioning,
each without and with Sorted representatives (1 per partition), sequential
final merge -- as one batch: every local skyline of the four queries in one
persistent engine launch, the four merges in a second.  The metric is input
points per second at the exact result (4 x N points per step).  Reported
beside it: the same four queries one at a time (`per_query_persistent`),
one at a time with one launch per partition (`plain`), the batch through the
C ABI from pinned host buffers (`e2e`), and a serving leg that replays a
Poisson arrival trace of mixed queries through the continuous-batching loop
and through the one-query-at-a-time plain path (p50/p99 latency).

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


from paper_2411_14968_gb300.replicas import dist_env  # noqa: E402


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


ENGINE_PROFILE = os.path.join(ROOT, "profiles", "k_engine_bench_ant1m_d6.txt")
ENGINE_SOURCE = os.path.join(ROOT, "paper_2411_14968_gb300", "csrc", "sky_engine_impl.cuh")


def engine_traffic():
    """DRAM bytes (read + write) of the engine launches of one batched step,
    from the committed ncu summary -- or None once the engine's source has
    changed since the counters were taken."""
    import hashlib
    if not os.path.exists(ENGINE_PROFILE):
        return None
    vals = {}
    with open(ENGINE_PROFILE) as fh:
        for ln in fh:
            if ln.startswith("# key ") and "=" in ln:
                k, v = ln[len("# key "):].strip().split("=", 1)
                vals[k.strip()] = v.strip()
    with open(ENGINE_SOURCE, "rb") as fh:
        src = hashlib.sha256(fh.read()).hexdigest()
    if vals.get("engine_source_sha256") != src or "dram_bytes_per_step" not in vals:
        return None
    return float(vals["dram_bytes_per_step"])


def load_workcounts():
    p = os.path.join(ROOT, "tests", "golden", "workcounts_ant_1m_d6.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        return json.load(fh)["variants"]


def host_cpu() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm
    implementer and part codes), with the core count."""
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            info = fh.read()
        for key in ("model name", "Model", "CPU part"):
            for ln in info.splitlines():
                if ln.split(":")[0].strip() == key:
                    model = f"{key}: {ln.split(':', 1)[1].strip()}"
                    break
            if model:
                break
    except OSError:
        pass
    return f"{model or 'unknown'}; {os.cpu_count()} logical cores"


def cpu_oracle_sample(n_sample: int, threads: int = 1):
    """Times the CPU oracle (C, as it stands) on the same variants over the
    first n_sample points of the same generator.  threads > 1 spreads
    Algorithm 2's local skylines over that many OpenMP threads (the merge
    stays sequential, as in the paper)."""
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
    O.set_threads(threads)
    try:
        t = time.perf_counter()
        for name, _ in VARIANTS:
            O.partitioned(x, **kw[name])
        return time.perf_counter() - t, len(VARIANTS) * n_sample
    finally:
        O.set_threads(1)


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
                         "sample": f"first {n_sample} points of the same generator, 4 variants per step",
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SERVE_QUERIES = 2000
SERVE_SEED = 5
SERVE_LOADS = (0.5, 0.8, 1.25, 4.0)  # offered load, x the plain path's measured capacity


def serving_pool(dev_pin: bool):
    """Seeded datasets the serving queries are drawn from: per (kind, d) one
    pool of 2^20 i.i.d. points; a query of N points is a window of N
    consecutive rows at a seeded offset.  The generators draw every row
    independently, so a window of N rows has exactly the distribution of a
    freshly generated N-point dataset of that kind and d; what windows do not
    give is independence between two queries whose windows overlap, which
    no per-query quantity measured here depends on.  Generating the 2,000
    queries' ~3e8 points one dataset at a time would take minutes."""
    import torch
    from paper_2411_14968_gb300 import datagen
    pool = {}
    for kind in ("anticorrelated", "independent"):
        for d in range(3, 9):
            if kind == "anticorrelated":
                x = datagen.anticorrelated(1 << 20, d, 900 + d)
            else:
                x = datagen.independent(1 << 20, d, 950 + d, quantised=False)
            t = torch.from_numpy(x)
            pool[(kind, d)] = t.pin_memory().numpy() if dev_pin else x
    return pool


def serving_queries(num: int, pool, native):
    from paper_2411_14968_gb300 import datagen
    rng = np.random.default_rng(SERVE_SEED)
    out = []
    for kind, n, d, _ in datagen.serving_trace(num, SERVE_SEED):
        base = pool[(kind, d)]
        off = int(rng.integers(0, base.shape[0] - n + 1))
        p = max(1, min(64, n // 8192))
        out.append((base[off: off + n], p))
    return out


def run_serving(ctx, native, queries, arrivals, exec_, workers, max_batch):
    """Replays the arrivals (seconds from start; None = all at once) through
    the serving loop; returns per-query latency (ms) and the makespan (s)."""
    ctx.serve_start(workers=workers, max_batch=max_batch)
    params = [native.make_params(scheme="sliced" if p > 1 else "none", p=p, exec=exec_) for _, p in queries]
    tickets = [None] * len(queries)
    t0 = time.perf_counter()
    for i, (x, _) in enumerate(queries):
        if arrivals is not None:
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
        tickets[i] = ctx.submit(x, params[i])
    lat, batch = [], []
    for t in tickets:
        _, info = ctx.wait(t)
        lat.append(info["latency_us"] / 1e3)
        batch.append(info["batch_queries"])
    span = time.perf_counter() - t0
    ctx.serve_stop()
    return np.array(lat), span, float(np.mean(batch))


def serving_leg(native, local, num_queries=SERVE_QUERIES):
    """Continuous batching vs one query at a time with one launch per
    partition, on the same Poisson arrival traces, at offered loads of 0.5,
    0.8, 1.25 and 4 x the plain path's measured capacity (the last one far
    beyond what the plain path serves, within what the batching loop does)."""
    from paper_2411_14968_gb300 import datagen
    pool = serving_pool(True)
    queries = serving_queries(num_queries, pool, native)
    total_pts = sum(x.shape[0] for x, _ in queries)
    ctx = native.Context(local)
    try:
        # warm-up of both forms on a few queries
        run_serving(ctx, native, queries[:8], None, "plain", 1, 1)
        run_serving(ctx, native, queries[:8], None, "persistent", 2, 64)
        # capacity of the plain one-at-a-time path (back-to-back)
        _, span_cap, _ = run_serving(ctx, native, queries, None, "plain", 1, 1)
        cap_qps = len(queries) / span_cap
        loads = []
        for load in SERVE_LOADS:
            rate = load * cap_qps
            arr = datagen.poisson_arrivals(len(queries), rate, SERVE_SEED)
            row = {"load": load, "offered_queries_per_s": rate}
            for name, exec_, w, mb in (("plain", "plain", 1, 1), ("batched", "persistent", 2, 64)):
                lat, span, mean_batch = run_serving(ctx, native, queries, arr, exec_, w, mb)
                row[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "mean_ms": float(lat.mean()), "points_per_s": total_pts / span,
                             "queries_per_s": len(queries) / span, "mean_batch_queries": mean_batch}
            loads.append(row)
        # saturation throughput of the batching loop (all queries at once)
        _, span_b, mb_sat = run_serving(ctx, native, queries, None, "persistent", 2, 64)
        res = {"loads": loads,
               "saturation": {"plain_points_per_s": total_pts / span_cap, "batched_points_per_s": total_pts / span_b,
                              "batched_mean_batch_queries": mb_sat},
               "plain_capacity_queries_per_s": cap_qps,
               "trace": (f"{len(queries)} queries of the 10,000-query serving trace (seed {SERVE_SEED}): "
                         "anticorrelated or independent FP32, N log-uniform in [1e3, 1e6], d uniform in 3..8, "
                         "Sliced p = clamp(N / 8192, 1, 64), each a window of a seeded 2^20-row pool of its kind "
                         "and d; Poisson arrivals at 0.5, 0.8, 1.25 and 4 x the measured capacity of the plain path "
                         "(the same arrival trace for both paths at each load)"),
               "points": total_pts}
        return res
    finally:
        ctx.close()


def serving_summary(serving):
    """p99 latency (ms) of both paths at each offered load."""
    if not serving:
        return None
    return {f"{row['load']}x": {"plain": round(row["plain"]["p99_ms"], 2),
                                 "batched": round(row["batched"]["p99_ms"], 2),
                                 "batched_mean_batch": round(row["batched"]["mean_batch_queries"], 2)}
            for row in serving["loads"]}


def gpu_arm(args, rank, world, local):
    import torch
    from paper_2411_14968_gb300 import datagen, native

    from paper_2411_14968_gb300.replicas import Replicas, throughput

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    reps = Replicas(world, dev)
    barrier, max_over_ranks = reps.barrier, reps.max_over_ranks

    x = datagen.anticorrelated(N, D, SEED)
    xt = torch.from_numpy(x).to(dev)
    ctx = native.Context(local)
    ctx.set_timing(True)
    tuning = None
    knobs = {}
    if not args.no_autotune:
        # the autotuner picks one set of engine knobs (SFS chunk sizes,
        # dominator block) for the batched step as a whole
        base = [(xt, native.make_params(**kw)) for _, kw in VARIANTS]
        ctx.skyline_batch(base)
        ctx.skyline_batch(base)
        default_ms = ctx.stats()["ms_total"]
        knobs, best_ms = ctx.autotune_batch(base, max_trials=40)
        tuning = {"tuned_on": "the batched step", "knobs": knobs, "default_knobs_ms": default_ms,
                  "tuned_ms": best_ms}
    persistent = {name: native.make_params(exec="persistent", **kw, **knobs) for name, kw in VARIANTS}
    plain = {name: native.make_params(exec="plain", **kw, **knobs) for name, kw in VARIANTS}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    names = [name for name, _ in VARIANTS]

    def step_batched(acc=None):
        # the four queries as one batch: every local skyline of the four in
        # one persistent launch, the four merges in a second one
        res = ctx.skyline_batch([(xt, persistent[nm]) for nm in names])
        if acc is not None:
            st = ctx.stats()
            acc["launches"] += st["launches"]
            acc["dom_ms"] += st["ms_dom_local"] + st["ms_dom_merge"]
            acc["stats"].append(st)
        return {nm: int(r.shape[0]) for nm, r in zip(names, res)}

    def step_each(pmap, acc=None):
        counts = {}
        for name, p in pmap.items():
            idx = ctx.skyline(xt, params=p)
            st = ctx.stats()
            counts[name] = int(idx.shape[0])
            if acc is not None:
                acc["launches"] += st["launches"]
                acc["dom_ms"] += st["ms_dom_local"] + st["ms_dom_merge"]
                acc["per_variant"].setdefault(name, []).append(st)
        return counts

    def timed(fn, k):
        acc = {"launches": 0, "dom_ms": 0.0, "per_variant": {}, "stats": []}
        ms = []
        barrier()
        torch.cuda.synchronize()
        for _ in range(k):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(acc)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier()
        return ms, acc

    # warm-up (also checks that every variant and form gives the same set:
    # Prop. 1)
    ref_counts = None
    for _ in range(max(args.warmup, 3)):
        c0 = step_batched()
        c1 = step_each(persistent)
        c2 = step_each(plain)
        if ref_counts is None:
            ref_counts = c1
        assert len(set(c0.values()) | set(c1.values()) | set(c2.values())) == 1, (c0, c1, c2)

    clocks = ClockSampler(local)
    clocks.start()
    ms, acc = timed(step_batched, args.steps)
    clk = clocks.stop()
    total_s = max_over_ranks(sum(ms) / 1e3)
    pts_per_step = N * len(VARIANTS)
    value = throughput(pts_per_step * args.steps, world, total_s)

    # the batched step captured into a CUDA graph and replayed
    graph = None
    if not args.no_graph:
        step_batched()
        batch_kernels = int(ctx.stats()["launches"])  # the graph holds the same kernels
        g = ctx.capture([(xt, persistent[nm]) for nm in names])
        for _ in range(max(args.warmup, 3)):
            res, _ = g.run()
            assert len({int(r.shape[0]) for r in res}) == 1
        gms = []
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between replays (before the replay's events)
            _, m_ = g.run()
            gms.append(m_)
        g_s = max_over_ranks(sum(gms) / 1e3)
        graph = {"value": throughput(pts_per_step * args.steps, world, g_s), "unit": "points/s",
                 "ms_per_step": sum(gms) / len(gms), "kernels_per_replay": batch_kernels,
                 "timing": "CUDA events around each replay on the graph's stream"}
        g.close()

    # one query at a time, every partition of a query in one launch
    ms_pq, acc_pq = timed(lambda a: step_each(persistent, a), max(1, args.steps))
    pq_value = pts_per_step * len(ms_pq) * world / max_over_ranks(sum(ms_pq) / 1e3)
    # plain form: one query at a time, one launch per partition
    ms_plain, acc_plain = timed(lambda a: step_each(plain, a), max(1, args.steps))
    plain_s = max_over_ranks(sum(ms_plain) / 1e3)
    plain_value = pts_per_step * len(ms_plain) * world / plain_s

    # end to end through the C ABI: pinned host inputs, host outputs
    xh = torch.from_numpy(x).pin_memory().numpy()
    sky_total = sum(ref_counts.values())
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k_e2e = max(1, args.steps)
    for _ in range(k_e2e):
        ctx.skyline_batch([(xh, persistent[nm]) for nm in names])
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = pts_per_step * k_e2e * world / e2e_s

    # roofline of the dominance kernel (k_engine): algorithmic compares
    # (oracle test count x d) over its measured launch time, against four
    # denominators: the derived FP32-compare peak (SMs x 64 compare lanes x
    # the maximum SM clock), the library's compare-rate probe (measured on
    # this GPU), the nominal ceiling of the instruction the hot loop issues
    # (sub.rn.f16x2 on 128 FMA lanes: one attribute of two tests per lane
    # per clock), and the library's rejection-loop probe (the engine's own
    # scan step run alone, measured on this GPU)
    wc = load_workcounts()
    roof = None
    dom_ms_per_step = acc["dom_ms"] / args.steps
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_ghz = (clk.get("sm_max_mhz") or 2070.0) / 1e3
    probe_tcmp = probe_reject = None
    try:
        rate, _ = ctx.probe_compare_rate()
        probe_tcmp = rate / 1e12
        rate, _ = ctx.probe_reject_rate()
        probe_reject = rate / 1e12
    except native.SkylineError:
        pass
    if wc:
        loc_ms = statistics.mean(st["ms_dom_local"] for st in acc["stats"])
        mer_ms = statistics.mean(st["ms_dom_merge"] for st in acc["stats"])
        t_loc = sum(wc[name]["local_tests"] for name in names)
        t_mer = sum(wc[name]["merge_tests"] for name in names)
        tests = t_loc + t_mer
        achieved = tests * D / (dom_ms_per_step * 1e-3) / 1e12
        peak = args.compare_peak_tcmp or sms * 64 * clk_ghz / 1e3
        f16 = sms * 128 * 2 * clk_ghz / 1e3
        a_loc = t_loc * D / (loc_ms * 1e-3) / 1e12
        a_mer = t_mer * D / (mer_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_engine (local + merge launches of the batched step)",
                "achieved": achieved, "peak": peak, "unit": "Tcmp/s", "frac": achieved / peak,
                "peak_source": f"derived: {sms} SMs x 64 FP32 compares/clk x {clk_ghz:.3f} GHz (max SM clock seen)",
                "peak_probe": probe_tcmp, "frac_probe": achieved / probe_tcmp if probe_tcmp else None,
                "f16x2_pipe_ceiling": f16, "frac_f16x2_pipe": achieved / f16,
                "f16x2_source": f"{sms} SMs x 128 FMA lanes x 2 dim-compares per sub.rn.f16x2 x {clk_ghz:.3f} GHz",
                "peak_reject_probe": probe_reject,
                "frac_reject_probe": achieved / probe_reject if probe_reject else None,
                "reject_probe_source": "sky_probe_reject_rate: the engine's f16x2 scan step alone, every test "
                                       "failing, 4 CTAs x 128 threads per SM, measured",
                "local": {"achieved": a_loc, "frac": a_loc / peak, "frac_f16x2_pipe": a_loc / f16,
                          "frac_reject_probe": a_loc / probe_reject if probe_reject else None,
                          "ms": loc_ms, "algorithmic_tests": t_loc},
                "merge": {"achieved": a_mer, "frac": a_mer / peak, "frac_f16x2_pipe": a_mer / f16,
                          "frac_reject_probe": a_mer / probe_reject if probe_reject else None,
                          "ms": mer_ms, "algorithmic_tests": t_mer},
                "engine_tests": {
                    "fp16": statistics.mean(st["tests_fp16"] for st in acc["stats"]),
                    "fp16_per_algorithmic_test": statistics.mean(st["tests_fp16"] for st in acc["stats"]) / tests,
                    "fp16_local": statistics.mean(st["tests_fp16_local"] for st in acc["stats"]),
                    "fp16_local_per_algorithmic_test":
                        statistics.mean(st["tests_fp16_local"] for st in acc["stats"]) / t_loc,
                    "fp16_merge_per_algorithmic_test":
                        statistics.mean(st["tests_fp16"] - st["tests_fp16_local"] for st in acc["stats"]) / t_mer,
                    "unit": "tests per step counted by the engine (candidate slots x staged dominators of its "
                            "16-bit test, dead slots included)"},
                "traffic": engine_traffic(), "traffic_unit": "DRAM bytes per step (ncu, both engine launches)",
                "algorithmic_tests_per_step": tests,
                "kernel_ms_per_step": dom_ms_per_step,
                "kernel_share_of_step": dom_ms_per_step / (sum(ms) / len(ms))}

    # per-variant breakdown of the one-query-at-a-time form (medians)
    per_variant = {}
    for name, sts in acc_pq["per_variant"].items():
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
    bst = acc["stats"][-1]
    batched_detail = {"ms_dom_local": bst["ms_dom_local"], "ms_dom_merge": bst["ms_dom_merge"],
                      "rounds_local": bst["rounds_local"], "rounds_merge": bst["rounds_merge"],
                      "ms_phase": [round(v, 4) for v in bst["ms_phase"]]}
    ctx.close()

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_leg(native, local, args.serve_queries)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_sample = 100_000
        secs, pts = cpu_oracle_sample(n_sample)
        cpu = {"value": pts / secs, "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n_sample} points of the same generator, the 4 variants once ({secs:.1f} s)",
               "host": host_cpu()}
        from oracle import oracle as O
        threads = min(O.max_threads(), os.cpu_count() or 1)
        if threads > 1:
            secs_mt, pts_mt = cpu_oracle_sample(n_sample, threads)
            cpu["parallel"] = {
                "value": pts_mt / secs_mt, "unit": "points/s", "cores": threads,
                "kind": "oracle with Algorithm 2's local skylines over OpenMP threads (sequential merge)",
                "sample": f"the same sample ({secs_mt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded anticorrelated generator; the paper's generator is unstated)",
            "config": {"workload": WORKLOAD, "points_per_step": pts_per_step,
                       "exec": "batched: the 4 queries in one call, all local skylines in one persistent launch, "
                               "all merges in a second",
                       "l2": "flushed between timed steps (256 MB write outside the timed events)",
                       "parallelism": f"replicas x{world}",
                       # the batched-vs-plain comparison of the metric, kept beside the headline
                       "plain_points_per_s": plain_value,
                       "speedup_batched_over_plain": value / plain_value,
                       "graph_points_per_s": graph["value"] if graph else None,
                       "serving_p99_ms": serving_summary(serving)},
            "graph": graph,
            "per_query_persistent": {"value": pq_value, "unit": "points/s",
                                     "ms_per_step": sum(ms_pq) / len(ms_pq)},
            "plain": {"value": plain_value, "unit": "points/s", "ms_per_step": sum(ms_plain) / len(ms_plain),
                      "speedup_batched_over_plain": value / plain_value},
            "e2e": {"value": e2e_value, "unit": "points/s",
                    "h2d_bytes_per_step": len(VARIANTS) * N * D * 4,
                    "d2h_bytes_per_step": 4 * sky_total + len(VARIANTS) * 128},
            "gpu_launches": int(acc["launches"]),
            "clocks": clk,
            "roofline": roof,
            "cpu_baseline": cpu,
            "serving": serving,
            "autotune": tuning,
            "batched": batched_detail,
            "variants": per_variant,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def rep_filtering_experiment(local: int):
    """Section 5 (Figure: effectiveness of representative filtering): the
    share of tuples that Sorted and Region representatives discard, on
    uniform, correlated and anticorrelated data with d = 4, under each
    partitioning scheme with 1 representative per partition."""
    import torch
    from paper_2411_14968_gb300 import datagen, native
    n, d = 1_000_000, 4
    data = {"uniform": datagen.independent(n, d, 41, quantised=False),
            "correlated": datagen.correlated(n, d, 42, quantised=False),
            "anticorrelated": datagen.anticorrelated(n, d, 43)}
    schemes = {"random": dict(scheme="random", p=64, seed=1), "grid": dict(scheme="grid", slices=[2] * d),
               "angular": dict(scheme="angular", slices=[4, 4, 4]), "sliced": dict(scheme="sliced", p=64)}
    out = {}
    with native.Context(local) as ctx:
        for dname, x in data.items():
            xt = torch.from_numpy(x).cuda()
            for sname, kw in schemes.items():
                row = {}
                sky = None
                for rep in ("sorted", "region"):
                    r = ctx.skyline(xt, params=native.make_params(rep=rep, grid_filter=False, **kw))
                    st = ctx.stats()
                    row[rep] = round(100.0 * st["rep_dropped"] / n, 2)
                    sky = int(r.shape[0]) if sky is None else sky
                    assert sky == int(r.shape[0])  # the result never depends on the representatives
                out[f"{dname}/{sname}"] = row
    print(json.dumps({"experiment": "representative filtering, % of tuples discarded (N=1e6, d=4, 1 rep per "
                                    "partition, Grid Filtering off)", "results": out}), flush=True)


def sweeps_experiment(local: int):
    """Section 5 (operating-parameter sweeps on anticorrelated data, defaults
    N = 1M, d = 4, p = 120): GPU time of the global skyline and the size of
    the local-skyline union for the plain strategies and the improved ones,
    varying N (1e5 to 1e8, the paper's range), d (2 to 7) and p (60 to
    3600) one at a time.  Grid and Angular reach p = 120 with per-dimension
    / per-angle slice counts (2,3,4,5) and (6,5,4).  Every result is
    compared with the oracle's skyline of the same input."""
    import torch
    from paper_2411_14968_gb300 import datagen, native

    def strategies(d, p):
        ang = {4: [6, 5, 4], 2: [p], 3: [12, 10]}.get(d)
        if ang is None:  # closest product to p with d - 1 factors of 2..6
            ang = [2] * (d - 1)
            i = 0
            while int(np.prod(ang)) * 2 <= p:
                ang[i % (d - 1)] += 1
                i += 1
        grid = [2, 3, 4, 5] if d == 4 else [2] * d
        return {
            "random": dict(scheme="random", p=p, seed=1), "grid": dict(scheme="grid", slices=grid),
            "angular": dict(scheme="angular", slices=ang), "sliced": dict(scheme="sliced", p=p),
            "sliced+": dict(scheme="sliced", p=p, rep="sorted"),
            "angular+": dict(scheme="angular", slices=ang, rep="sorted"),
            "noseq": dict(scheme="sliced", p=p, rep="sorted", merge="noseq"),
        }

    import hashlib
    gold_path = os.path.join(ROOT, "tests", "golden", "sweep_skylines.json")
    gold = json.load(open(gold_path)) if os.path.exists(gold_path) else {}
    rows = []
    with native.Context(local) as ctx:
        ctx.set_timing(True)

        def run(n, d, seed, p, names, tag):
            # every result is checked against the oracle's skyline of the same
            # input (|Sky| and SHA-256 of the ascending indices, written by
            # tests/golden/make_sweeps.py)
            x = datagen.anticorrelated_blocks(n, d, seed)
            g = gold.get(f"n={n},d={d},seed={seed}")
            if g:
                assert hashlib.sha256(x.astype("<f4").tobytes()).hexdigest() == g["input_sha256"], (n, d, seed)
            xt = torch.from_numpy(x).cuda()
            del x
            strat = strategies(d, p)
            for name in names:
                pr = native.make_params(**strat[name])
                ctx.skyline(xt, params=pr)  # warm-up (workspace)
                ms = []
                for _ in range(2):
                    r = ctx.skyline(xt, params=pr)
                    ms.append(ctx.stats()["ms_total"])
                st = ctx.stats()
                idx = r.cpu().numpy().astype("<u4")
                match = None
                if g:
                    match = (idx.shape[0] == g["skyline"] and
                             hashlib.sha256(idx.tobytes()).hexdigest() == g["skyline_sha256"])
                    assert match, (tag, n, d, p, name)
                rows.append({"sweep": tag, "n": n, "d": d, "p": st["partitions"], "strategy": name,
                             "ms": round(min(ms), 3), "local_union": st["local_union"], "skyline": int(idx.shape[0]),
                             "points_per_s": n / (min(ms) * 1e-3), "oracle_match": match})
                print(json.dumps(rows[-1]), flush=True)
            del xt
            torch.cuda.empty_cache()

        plain = ["random", "grid", "angular", "sliced"]
        improved = ["sliced+", "angular+", "noseq"]
        for n in (100_000, 500_000, 1_000_000, 5_000_000, 10_000_000, 50_000_000, 100_000_000):
            run(n, 4, 7, 120, plain + improved, "size")
        for d in (2, 3, 5, 6, 7):
            run(1_000_000, d, 8, 120, improved, "dimensions")
        for p in (60, 240, 480, 720, 1200, 2400, 3600):
            run(1_000_000, 4, 7, p, ["sliced+", "noseq"], "partitions")
    print(json.dumps({"experiment": "sweeps (anticorrelated; defaults N=1e6, d=4, p=120)", "rows": rows}), flush=True)


def configs_experiment(local: int):
    """Throughput of the other workload configurations (points per second,
    one query at a time and as one batch, CUDA events), beside the headline
    one: the tiny Grid case; 4M-point d = 8 quantised independent and
    correlated data, Grid m = 2 (256 cells) vs Random p = 256; 2M-point
    skewed record-like data, Angular p = 128 with Sorted representatives,
    NoSeq vs the sequential final phase."""
    import torch
    from paper_2411_14968_gb300 import datagen, native
    cases = [
        ("anticorrelated N=1e4 d=4, Grid m=2 (16 cells)", ("anticorrelated", 10_000, 4, 1),
         [dict(scheme="grid", slices=[2] * 4)]),
        ("independent quantised N=4e6 d=8, Grid m=2 vs Random p=256", ("independent", 4_000_000, 8, 3),
         [dict(scheme="grid", slices=[2] * 8), dict(scheme="random", p=256, seed=11)]),
        ("correlated quantised N=4e6 d=8, Grid m=2 vs Random p=256", ("correlated", 4_000_000, 8, 3),
         [dict(scheme="grid", slices=[2] * 8), dict(scheme="random", p=256, seed=11)]),
        ("skewed N=2e6 d=6, Angular (4,4,2,2,2) + Sorted reps, sequential vs NoSeq", ("skewed", 2_000_000, 6, 4),
         [dict(scheme="angular", slices=[4, 4, 2, 2, 2], normalize=True, rep="sorted"),
          dict(scheme="angular", slices=[4, 4, 2, 2, 2], normalize=True, rep="sorted", merge="noseq")]),
    ]
    out = []
    wc_path = os.path.join(ROOT, "tests", "golden", "workcounts_skewed_2m_d6.json")
    skewed_wc = json.load(open(wc_path))["variants"]["angular_rep"] if os.path.exists(wc_path) else None
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    with native.Context(local) as ctx:
        ctx.set_timing(True)
        for title, (kind, n, d, seed), variants in cases:
            xt = torch.from_numpy(datagen.make(kind, n, d, seed)).cuda()
            row = {"config": title, "variants": []}
            for kw in variants:
                p = native.make_params(**kw)
                ctx.skyline(xt, params=p)
                ms = []
                for _ in range(3):
                    r = ctx.skyline(xt, params=p)
                    ms.append(ctx.stats()["ms_total"])
                st = ctx.stats()
                v = {"params": kw, "ms": round(min(ms), 3), "points_per_s": n / (min(ms) * 1e-3),
                     "skyline": int(r.shape[0]), "local_union": st["local_union"],
                     "ms_dom_local": round(st["ms_dom_local"], 3), "ms_dom_merge": round(st["ms_dom_merge"], 3)}
                if kind == "skewed" and kw.get("merge", "sequential") == "sequential" and skewed_wc:
                    # compare-pipe roofline of the engine on this workload: the
                    # oracle's SFS test count x d over the two engine launches
                    t = skewed_wc["local_tests"] + skewed_wc["merge_tests"]
                    dom = st["ms_dom_local"] + st["ms_dom_merge"]
                    peak = sms * 64 * 2.07e9
                    v["roofline"] = {"algorithmic_tests": t, "achieved_tcmp": t * d / (dom * 1e-3) / 1e12,
                                     "frac_of_derived_fp32_peak": t * d / (dom * 1e-3) / peak}
                row["variants"].append(v)
            if len(variants) > 1:
                ps = [native.make_params(**kw) for kw in variants]
                ctx.skyline_batch([(xt, p) for p in ps])
                bms = []
                for _ in range(3):
                    ctx.skyline_batch([(xt, p) for p in ps])
                    bms.append(ctx.stats()["ms_total"])
                row["batched"] = {"ms": round(min(bms), 3),
                                  "points_per_s": n * len(variants) / (min(bms) * 1e-3)}
            out.append(row)
            print(json.dumps(row), flush=True)
    print(json.dumps({"experiment": "workload configurations", "rows": out}), flush=True)


def shapes_experiment(local: int):
    """The batched step (the benchmark's four queries as one batch) with each
    compiled launch shape of the engine -- warps per CTA x candidates per
    lane, i.e. the tile width of a work item -- at the default chunk and
    block knobs: device time of the whole batch and of its two engine
    launches (median of 7 runs, CUDA events)."""
    import torch
    from paper_2411_14968_gb300 import datagen, native
    x = datagen.anticorrelated(N, D, SEED)
    xt = torch.from_numpy(x).cuda()
    rows = []
    with native.Context(local) as ctx:
        ctx.set_timing(True)
        for w, r in ((4, 4), (8, 4), (4, 2), (8, 2)):
            ps = [native.make_params(engine_warps=w, engine_cands=r, **kw) for _, kw in VARIANTS]
            for _ in range(2):
                ctx.skyline_batch([(xt, p) for p in ps])
            sts = []
            for _ in range(7):
                ctx.skyline_batch([(xt, p) for p in ps])
                sts.append(ctx.stats())
            med = lambda k: statistics.median(st[k] for st in sts)  # noqa: E731
            rows.append({"warps": w, "cands_per_lane": r, "tile": 32 * w * r, "ms_total": round(med("ms_total"), 3),
                         "ms_dom_local": round(med("ms_dom_local"), 3), "ms_dom_merge": round(med("ms_dom_merge"), 3),
                         "points_per_s": len(VARIANTS) * N / (med("ms_total") * 1e-3)})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"experiment": "engine launch shapes on the batched step", "rows": rows}), flush=True)


VALUE_RANGES = [
    ("unit [0,1]", 1.0, 0.0),
    ("offset +1024", 1.0, 1024.0),
    ("scaled x2^17", 2.0 ** 17, 0.0),
    ("scaled x2^-20", 2.0 ** -20, 0.0),
]


def value_range_experiment(local: int):
    """The batched step (the benchmark's four queries on one input) on the
    benchmark's anticorrelated points moved into other value ranges (scaled
    by a power of two, which keeps every comparison; or offset, where FP32
    rounding makes some values equal), with the FP16 images of the values
    and with the rank images (sky_rank_space): device time of the batch and
    of its two engine launches, median of 7 runs.  Each range's skyline is
    checked against the oracle once (its threaded Algorithm 2: Sliced p=64
    with the NoSeq merge, whose skyline equals sequential SFS's)."""
    import torch
    from paper_2411_14968_gb300 import datagen, native
    from oracle import oracle as O
    O.set_threads(os.cpu_count() or 1)
    x0 = datagen.anticorrelated(N, D, SEED)
    rows = []
    with native.Context(local) as ctx:
        ctx.set_timing(True)
        for name, scale, offset in VALUE_RANGES:
            x = np.ascontiguousarray(x0 * np.float32(scale) + np.float32(offset), dtype=np.float32)
            want = O.partitioned(x, scheme=O.SLICED, p=64, merge=O.MERGE_NOSEQ)["indices"]
            xt = torch.from_numpy(x).cuda()
            for images in ("values", "ranks"):
                ps = [native.make_params(images=images, **kw) for _, kw in VARIANTS]
                for _ in range(2):
                    got = ctx.skyline_batch([(xt, p) for p in ps])
                for g in got:
                    assert np.array_equal(g.cpu().numpy().astype(np.uint32), want), (name, images)
                sts = []
                for _ in range(7):
                    ctx.skyline_batch([(xt, p) for p in ps])
                    sts.append(ctx.stats())
                med = lambda k: statistics.median(st[k] for st in sts)  # noqa: E731
                rows.append({"values": name, "images": images, "skyline": int(want.shape[0]),
                             "ms_total": round(med("ms_total"), 3), "ms_prep": round(sts[0]["ms_phase"][0], 3),
                             "ms_dom_local": round(med("ms_dom_local"), 3),
                             "ms_dom_merge": round(med("ms_dom_merge"), 3),
                             "points_per_s": len(VARIANTS) * N / (med("ms_total") * 1e-3)})
                print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"experiment": "value ranges: FP16 images of the values vs rank images", "rows": rows}),
          flush=True)


def fp16_images(x):
    """Round-down FP16 images of FP32 values, clamped to the finite FP16
    range (the images the dominance kernels test first)."""
    h = x.astype(np.float16)
    down = h.astype(np.float32) > x
    h[down] = np.nextafter(h[down], np.float16(-np.inf))
    return np.clip(h, np.float16(-65504.0), np.float16(65504.0))


def fp16_experiment():
    """How often the FP16 test passes a pair that Def. 1 then rejects, on
    each workload's data (host-side, numpy): 3000 x 3000 sampled pairs (s, t)
    with score(s) <= score(t); pass = every image of s <= t's, dominates =
    Def. 1 on the FP32 values.  pass & not dominates is the FP32 work the
    images cannot save (ties of images, or of the values themselves)."""
    from paper_2411_14968_gb300 import datagen
    rng = np.random.default_rng(3)
    cases = [("anticorrelated N=1e6 d=6", datagen.anticorrelated(1_000_000, 6, 1)),
             ("independent quantised N=4e6 d=8", datagen.independent(4_000_000, 8, 3)),
             ("skewed N=2e6 d=6", datagen.skewed(2_000_000, 6, 4))]
    out = []
    for name, x in cases:
        idx = rng.choice(x.shape[0], 3000, replace=False)
        jdx = rng.choice(x.shape[0], 3000, replace=False)
        t, sp = x[idx], x[jdx]
        ht, hs = fp16_images(t), fp16_images(sp)
        ft = t.astype(np.float32).sum(axis=1, dtype=np.float32)
        fs = sp.astype(np.float32).sum(axis=1, dtype=np.float32)
        order = fs[:, None] <= ft[None, :]
        pas = np.ones((3000, 3000), bool)
        le = np.ones((3000, 3000), bool)
        ne = np.zeros((3000, 3000), bool)
        for k in range(x.shape[1]):
            pas &= hs[:, k][:, None] <= ht[:, k][None, :]
            le &= sp[:, k][:, None] <= t[:, k][None, :]
            ne |= sp[:, k][:, None] != t[:, k][None, :]
        dom = le & ne & order
        pas &= order
        npairs = int(order.sum())
        row = {"workload": name, "pairs": npairs, "fp16_pass": float(pas.sum() / npairs),
               "dominates": float(dom.sum() / npairs),
               "pass_not_dominates": float((pas & ~dom).sum() / npairs),
               "fp32_checks_per_kill": float(pas.sum() / max(1, dom.sum()))}
        out.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"experiment": "FP16 image test vs Def. 1 on sampled pairs", "rows": out}), flush=True)


def ncu_case(which: str):
    """The cases the engine's ncu captures run: the two k_engine launches
    (local phase, merge) of the second call are the captured ones."""
    import torch
    from paper_2411_14968_gb300 import datagen, native
    if which == "noseq":
        # one skewed query, N = 200k, d = 6, Angular (4,4,2,2,2) + Sorted
        # reps, NoSeq final phase: the NoSeq kernel's profile case
        x = datagen.skewed(200_000, 6, 4)
        xt = torch.from_numpy(x).cuda()
        with native.Context(0) as ctx:
            p = native.make_params(scheme="angular", slices=[4, 4, 2, 2, 2], normalize=True, rep="sorted",
                                   merge="noseq")
            for _ in range(2):
                r = ctx.skyline(xt, params=p)
            torch.cuda.synchronize()
            print(f"ncu case noseq: |Sky| = {r.shape[0]}, {ctx.stats()['launches']} launches per call")
        return
    if which == "rank":
        # rank space of 4M anticorrelated points, d = 8 (128 MB of input):
        # the rank kernels and the sorts of sky_rank_space, per column
        x = datagen.anticorrelated(4_000_000, 8, 3)
        xt = torch.from_numpy(x).cuda()
        with native.Context(0) as ctx:
            ctx.set_timing(True)
            for _ in range(2):
                r, dist, _ = ctx.rank_space(xt)
            torch.cuda.synchronize()
            st = ctx.stats()
            print(f"ncu case rank: distinct {dist.cpu().tolist()}, {st['launches']} launches, "
                  f"{st['ms_total']:.3f} ms per call")
        return
    if which == "c3":
        # one 4M-point d = 8 quantised independent query, Grid m = 2 (256
        # cells): the workload where the memory-bound stages bound the query
        x = datagen.independent(4_000_000, 8, 3)
        xt = torch.from_numpy(x).cuda()
        with native.Context(0) as ctx:
            p = native.make_params(scheme="grid", slices=[2] * 8)
            for _ in range(2):
                r = ctx.skyline(xt, params=p)
            torch.cuda.synchronize()
            print(f"ncu case c3: |Sky| = {r.shape[0]}, {ctx.stats()['launches']} launches per call")
        return
    n = 200_000 if which == "small" else N
    x = datagen.anticorrelated(n, D, SEED)
    xt = torch.from_numpy(x).cuda()
    with native.Context(0) as ctx:
        if which == "small":
            p = native.make_params(scheme="sliced", p=64)
            for _ in range(2):
                r = ctx.skyline(xt, params=p)
        else:
            ps = [native.make_params(**kw) for _, kw in VARIANTS]
            for _ in range(2):
                r = ctx.skyline_batch([(xt, p) for p in ps])[0]
        torch.cuda.synchronize()
        print(f"ncu case {which}: |Sky| = {r.shape[0]}, {ctx.stats()['launches']} launches per call")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--experiment", choices=["rep-filtering", "sweeps", "configs", "shapes", "fp16", "value-range"],
                    default=None,
                    help="run one of the paper's experiments instead of the benchmark")
    ap.add_argument("--ncu-case", choices=["small", "batch", "c3", "noseq", "rank"], default=None,
                    help="run a profiling case only, twice, default knobs, no timing: 'small' = one query "
                         "(anticorrelated N=200k, d=6, Sliced p=64); 'batch' = the benchmark's batched step; "
                         "'c3' = one quantised independent query, N=4M, d=8, Grid m=2; 'noseq' = one skewed "
                         "query, N=200k, d=6, Angular (4,4,2,2,2) + Sorted reps, NoSeq; 'rank' = sky_rank_space "
                         "of 4M anticorrelated points, d=8")
    # FP32 compare peak in T compares/s; 0 derives it from the device's SM
    # count x 64 compare lanes per SM per clock x the maximum SM clock seen
    ap.add_argument("--compare-peak-tcmp", type=float, default=0.0)
    ap.add_argument("--serve-queries", type=int, default=SERVE_QUERIES)
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.ncu_case:
        ncu_case(args.ncu_case)
        return
    if args.experiment == "rep-filtering":
        rep_filtering_experiment(local)
        return
    if args.experiment == "sweeps":
        sweeps_experiment(local)
        return
    if args.experiment == "configs":
        configs_experiment(local)
        return
    if args.experiment == "shapes":
        shapes_experiment(local)
        return
    if args.experiment == "fp16":
        fp16_experiment()
        return
    if args.experiment == "value-range":
        value_range_experiment(local)
        return
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    gpu_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
