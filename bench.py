"""Benchmark: PG-SGD layout updates/s on the 5 M-node synthetic chromosome graph.

One step = one whole layout of the graph (Algorithm 1: 30 iterations of
10 x S lock-free updates, S = total path steps) followed by its sampled path
stress (Eq. 2, 100 samples per step), starting every step from the same
initial layout. Inputs are resident in HBM when the timed region starts
(3.9 GB of packed records: larger than L2, so no flush is needed).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config chrom|mid|tiny]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Multi-GPU: the layout does not shard (every path crosses the shared backbone),
so N > 1 runs N independent replicas, one per GPU, under torchrun; the line
reports their aggregate throughput ("weak" scaling, no collective on the data
path: the process group only times the replicas).
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

METRIC = "PG-SGD updates/sec and % HBM roofline on 5M-node graph; stress vs oracle"
UNIT = "updates/s"
ITERS = 30
THETA = 0.99
SEED = 1
STRESS_PER_STEP = 100
STRESS_SEED = 7
# DRAM sectors an update touches with no cache reuse: 2 step-record sectors and
# 2 node-record sectors read, 2 node-record sectors written back (32 B each).
BYTES_PER_UPDATE = 192
WORKLOADS = {
    "chrom": "synthetic chromosome-scale pangenome: 5,000,000 backbone nodes (+10% bubble "
             "nodes), 90 paths, ~4.7e8 steps, node length geometric mean 30 bp with a 1e-4 "
             "tail to 100 kb; 30 iterations x 10 x steps updates; theta 0.99",
    "mid": "synthetic pangenome: 200,000 backbone nodes, 32 paths, ~7e6 steps",
    "tiny": "synthetic pangenome: 2,000 backbone nodes, 8 paths, ~1.6e4 steps",
    "prof": "synthetic chromosome-like pangenome for profiling: 2,000,000 backbone nodes, "
            "30 paths, ~6.3e7 steps (0.6 GB on device, above L2)",
    "batch256": "256 independent synthetic subgraphs, node counts log-uniform in [1,000, 200,000], "
                "path counts uniform in [4, 90] (8.6e6 nodes, 4.0e8 steps in all); 30 iterations "
                "x 10 x steps updates per graph, each graph with its own learning-rate schedule",
    "batch_prof": "64 independent synthetic subgraphs drawn like batch256 (profiling case, ~1.5 GB)",
}
BATCH_WORKLOADS = ("batch256", "batch_prof")
BATCH_METRIC = "PG-SGD updates/sec, batched layout of 256 subgraphs (one persistent or CUDA-graph launch " \
               "sequence) vs one launch per graph; per-graph stress"


# ---------------------------------------------------------------- distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return ws, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_rate(units: float, ms: float, device=None) -> float:
    """Whole-job rate: the units all ranks processed / the slowest rank's time."""
    return sum_over_ranks(units, device) / (max_over_ranks(ms, device) / 1e3)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap", "timestamp"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Clock record of the timed region from nvidia-smi CSV samples (the fields
    of ClockSampler.FIELDS): median SM clock over the loaded samples (those at
    least half the highest), the maximum clock, and every throttle reason seen
    active in any sample."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 8:  # the timestamp (field 9) is not needed here
            continue
        try:
            sm.append(float(parts[0]))
            smax.append(float(parts[1]))
        except ValueError:
            continue
        for name, val in zip(names, parts[4:8]):
            if val.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    top = max(sm)
    loaded = [s for s in sm if s >= 0.5 * top] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
            "reasons": sorted(reasons), "samples": len(sm)}


def _sample_time(field):
    """Epoch seconds of an nvidia-smi timestamp ("2026/12/04 06:12:34.567", local time)."""
    from datetime import datetime
    try:
        return datetime.strptime(field.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
    except ValueError:
        return None


def clocks_in_windows(lines, windows):
    """Median SM clock and power of the samples taken inside the host-time
    windows [(t0, t1), ...] (epoch seconds): the clock a phase ran at."""
    sm, pw = [], []
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < len(ClockSampler.FIELDS):
            continue
        t = _sample_time(parts[8])
        if t is None or not any(a <= t <= b for a, b in windows):
            continue
        try:
            sm.append(float(parts[0]))
            pw.append(float(parts[2]))
        except ValueError:
            continue
    if not sm:
        return {"sm_mhz_median": None, "samples": 0}
    return {"sm_mhz_median": statistics.median(sm), "sm_mhz_min": min(sm), "power_w_median": statistics.median(pw),
            "samples": len(sm)}


# ---------------------------------------------------------------- workload

def make_workload(config):
    from synth import BATCH_CONFIGS, batch_shapes, make_batch, make_graph
    if config in BATCH_CONFIGS:
        # the oracle's bounded sample runs on the batch's largest graph
        cfg = BATCH_CONFIGS[config]
        shapes = batch_shapes(cfg["n_graphs"], cfg["nodes"], cfg["paths"], cfg["seed"])
        k = max(range(len(shapes)), key=lambda i: shapes[i][0] * shapes[i][1])
        return make_batch(config, indices=[k])[0]
    if config == "prof":
        return make_graph("chrom", backbone=2_000_000, paths=30)
    return make_graph(config)


def workload_config(name, n_nodes, n_paths, n_steps, ws):
    """The `config` object of both arms' lines: the workload and its sizes
    (the same for the GPU arm and the oracle arm), and how L2 is handled
    between timed steps: the 16-byte step records alone exceed L2, so no flush."""
    return {"workload": WORKLOADS[name], "name": name, "n_nodes": int(n_nodes), "n_paths": int(n_paths),
            "n_steps": int(n_steps), "iterations": ITERS, "updates_per_step": ITERS * 10 * int(n_steps),
            "stress_samples_per_step": STRESS_PER_STEP * int(n_steps),
            "l2": f"inputs larger than L2 ({16 * n_steps / 1e9:.1f} GB of step records), no flush",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _oracle_rate(g, eta, t, budget_s, threads):
    """Updates/s of the oracle's Hogwild! mode on the first updates of
    iteration t, sized to take about budget_s (a probe sizes the sample)."""
    import oracle as O
    probe = max(100_000, min(g.n_steps, 2_000_000))
    t0 = time.perf_counter()
    O.layout(g, g.init_xy, T=ITERS, eta=eta, theta=THETA, seed=SEED, t_begin=t, t_end=t + 1, n_updates=probe,
             n_threads=threads)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    n = int(min(max(rate * budget_s, probe), 10 * g.n_steps))
    t0 = time.perf_counter()
    O.layout(g, g.init_xy, T=ITERS, eta=eta, theta=THETA, seed=SEED, t_begin=t, t_end=t + 1, n_updates=n,
             n_threads=threads)
    return n, time.perf_counter() - t0


def cpu_baseline(g, budget_s=12.0, warmup=False):
    """The oracle (threaded Hogwild! mode, all host cores) on bounded samples
    of the same workload: the first updates of a mixed iteration (t = 2: half
    uniform, half power-law partners) and of a cooling iteration (t = 20: all
    power-law partners, with their rejection trials), about budget_s / 2 each.
    The rate is updates / time over both samples; a whole layout has 15
    iterations of each kind, so this weights them as the layout does."""
    import oracle as O
    threads = os.cpu_count() or 1
    eta = O.eta_schedule(ITERS, O.default_eta_max(g))
    parts = {t: _oracle_rate(g, eta, t, budget_s / 2, threads) for t in (2, 20)}
    n = sum(v[0] for v in parts.values())
    dt = sum(v[1] for v in parts.values())
    desc = ", ".join(f"t = {t}: first {v[0]} updates ({v[0] / (10 * g.n_steps):.2%} of the iteration) in "
                     f"{v[1]:.1f} s = {v[0] / v[1]:.3g} upd/s" for t, v in parts.items())
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "per_iteration_kind": {"mixed_t2": parts[2][0] / parts[2][1], "cooling_t20": parts[20][0] / parts[20][1]},
            "sample": f"bounded samples of the same graph and seed, FP64, {threads} threads: {desc}"}


def cpu_full_layouts(names=("tiny",), single_thread=("tiny",)):
    """Whole oracle layouts (30 iterations x 10 x S updates) timed on the host:
    all cores (Hogwild!), and one thread (the sequential definition) for the
    workloads in single_thread."""
    import oracle as O
    from synth import make_graph
    threads = os.cpu_count() or 1
    out = {}
    for name in names:
        g = make_graph(name)
        eta = O.eta_schedule(ITERS, O.default_eta_max(g))
        row = {"updates": ITERS * 10 * g.n_steps}
        for k in sorted({1, threads} if name in single_thread else {threads}):
            t0 = time.perf_counter()
            O.layout(g, g.init_xy, T=ITERS, eta=eta, theta=THETA, seed=SEED, n_threads=k)
            dt = time.perf_counter() - t0
            row[f"threads_{k}"] = {"seconds": dt, "updates_per_s": row["updates"] / dt}
        out[name] = row
    return out


def stress_vs_oracle(G, config):
    """The layout's sampled stress (Eq. 2) against the oracle's layouts of the
    same graph under the same layout seed, on the same sample set (the stored
    record's samples per step and stress seed; tests/golden/oracle_layouts.json,
    written by tests/golden/make_oracle_layouts.py)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_layouts.json")
    if not os.path.exists(path):
        return None
    data = json.load(open(path))
    # prefer the record with the larger sample set where there is one (reading: the
    # 200 k-node graph's stress at 100 samples per step is dominated by its sample set)
    name = f"{config}_1000" if f"{config}_1000" in data else config
    rec = data.get(name)
    if not rec:
        return None
    runs = [r for r in rec["runs"] if r["seed"] == SEED]
    if not runs:
        return None
    st = G.stress(rec["stress_samples_per_step"], seed=rec["stress_seed"])
    ref = np.array([r["stress"] for r in runs])
    out = {"record": name, "samples_per_step": rec["stress_samples_per_step"], "stress_seed": rec["stress_seed"],
           "layout_seed": SEED, "gpu_mean": st["mean"], "gpu_ci": [st["ci_lo"], st["ci_hi"]],
           "oracle_mean": float(ref.mean()), "oracle_runs": len(ref), "oracle_threads": rec["oracle_threads"],
           "oracle_ci_first_run": [runs[0]["ci_lo"], runs[0]["ci_hi"]],
           "ratio": st["mean"] / float(ref.mean())}
    if len(ref) > 1:
        out["oracle_run_to_run_rel_sd"] = float(ref.std(ddof=1) / ref.mean())
    return out


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    g = make_workload(args.config)
    import oracle as O
    O.build()
    for _ in range(args.warmup):
        cpu_baseline(g, budget_s=args.ref_budget)
    vals = [cpu_baseline(g, budget_s=args.ref_budget) for _ in range(args.steps)]
    value = statistics.mean(v["value"] for v in vals)
    cb = dict(vals[-1])
    cb["value"] = value
    updates_per_step = ITERS * 10 * g.n_steps
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": updates_per_step / value * 1e3, "higher_is_better": True,
        "ms_per_step_extrapolated": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.config, g.n_nodes, g.n_paths, g.n_steps, args.gpus),
        "sample": "each step times bounded samples of a mixed (t = 2) and a cooling (t = 20) "
                  "iteration (see cpu_baseline); ms_per_step is one whole layout's updates at "
                  "that rate, extrapolated, not timed",
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_dist("nccl" if ws > 1 else "gloo")
    dev = torch.device("cuda", local)
    import paper_2409_00876_gb300 as pg
    pg.load_library()

    g = make_workload(args.config)
    xy0 = torch.from_numpy(g.init_xy).to(dev)
    G = pg.Graph.from_synth(g)
    G.set_coords(xy0)
    info = G.info()
    S = info["n_steps"]
    updates_per_step = ITERS * 10 * S
    stream = torch.cuda.current_stream()

    windows = {"layout": [], "stress": []}
    phase_events = []

    def step(timed=False):
        t0 = time.time()
        G.set_coords(xy0)
        G.layout(ITERS, theta=THETA, seed=SEED)
        if timed:
            # phase boundary: host time for the clock record, an event for the device time
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            stream.synchronize()
            t1 = time.time()
        st = G.stress(STRESS_PER_STEP, seed=STRESS_SEED)  # synchronous
        if timed:
            ev2 = torch.cuda.Event(enable_timing=True)
            ev2.record(stream)
            windows["layout"].append((t0, t1))
            windows["stress"].append((t1, time.time()))
            phase_events.append((ev, ev2))
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    G.set_option("timing", 1)
    G.timing_read(reset=True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = None
    for _ in range(args.steps):
        st = step(timed=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    upd_ms, launches, upd = G.timing_read(reset=True)
    G.set_option("timing", 0)
    stress_ms = [a.elapsed_time(b) for a, b in phase_events]
    n_samples = STRESS_PER_STEP * S
    phases = {"layout": {"update_launch_ms_per_step": upd_ms / args.steps,
                         **clocks_in_windows(clocks.lines, windows["layout"])},
              "stress": {"ms_per_step": statistics.mean(stress_ms), "ms_each": [round(x, 1) for x in stress_ms],
                         "samples_per_s": n_samples / (statistics.mean(stress_ms) / 1e3),
                         **clocks_in_windows(clocks.lines, windows["stress"])}}
    ph = phases["stress"]
    if ph.get("sm_mhz_median"):
        # time x clock: equal across GPUs when a difference in time is a difference in clock
        ph["ms_x_ghz"] = ph["ms_per_step"] * ph["sm_mhz_median"] / 1e3
    vs_oracle = stress_vs_oracle(G, args.config) if rank == 0 else None
    # the stress kernel makes the same random reads as an update (two step
    # records, two node points) with no arithmetic of note and no writes: its
    # rate on this GPU is the measured gather rate the update kernel is held to
    gather_ref = {"kernel": "stress_kernel (Eq. 2): the same two random step-record reads and two node reads "
                            "per unit, no moves, no writes", "units_per_s": phases["stress"]["samples_per_s"]}
    ms_max = max_over_ranks(ms, dev)
    value = aggregate_rate(updates_per_step * args.steps, ms, dev)

    # kernels launched per step: set_coords + anchor refresh, 30 x (update +
    # rebase + anchor refresh), stress + finalize
    gpu_launches = args.steps * (2 + 3 * ITERS + 2)
    peak, peak_kind = peaks()
    per_launch_ms = upd_ms / max(launches, 1)
    updates_per_launch = upd / max(launches, 1)
    achieved = BYTES_PER_UPDATE * updates_per_launch / (per_launch_ms / 1e3) / 1e9
    gather = hbm_gather(pg) if args.config in ("chrom", "prof") and not args.skip_gather else None
    # ncu DRAM bytes per update, captured on the 2 M-node profiling graph (the same
    # record sizes and access pattern, 1 GB resident) and scaled to this launch's updates
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "update_kernel_traffic_prof.json")
    if os.path.exists(tpath) and args.config in ("chrom", "prof"):
        tr = json.load(open(tpath))
        if tr.get("kernel_rev") == kernel_revision():
            traffic = tr["dram_bytes_per_update"] * updates_per_launch

    # end to end through the public API with host buffers, copies inside the region
    e2e = run_e2e(pg, g, args, dev) if not args.skip_e2e else None
    if e2e is not None:
        e2e["value"] = aggregate_rate(e2e.pop("updates"), 1e3 * e2e.pop("seconds"), dev)

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = cpu_baseline(g, budget_s=args.cpu_budget)
        cpu["full_layouts"] = cpu_full_layouts(tuple(args.cpu_full))

    forms = None
    if rank == 0 and not args.no_forms and args.config == "chrom":
        forms = {"data_reuse": reuse_form(G, xy0), "batched": batch_form(dev),
                 "differentiable": dstress_form(dev)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.config, info["n_nodes"], info["n_paths"], S, ws),
            "device_bytes": info["device_bytes"],
            "stress": {"mean": st["mean"], "ci_lo": st["ci_lo"], "ci_hi": st["ci_hi"],
                       "n_valid": st["n_valid"]},
            "layout_only_updates_per_s": upd / (upd_ms / 1e3) if upd_ms > 0 else None,
            "stress_vs_oracle": vs_oracle,
            "roofline": roofline_for(args.config, achieved, peak, peak_kind, traffic, per_launch_ms, gather,
                                     2 * updates_per_launch / (per_launch_ms / 1e3), gather_ref,
                                     updates_per_launch / (per_launch_ms / 1e3)),
            "clocks": clk,
            "phases": phases,
            "gpu_launches": gpu_launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- batched and differentiable forms

def _batch_timed(B, xy, seeds, iter_end=None):
    """Milliseconds of one full layout from xy (library events on the stream)."""
    B.set_coords(xy)
    B.set_option("timing", 1)
    B.timing_read(reset=True)
    B.layout(ITERS, seeds=seeds, theta=THETA, iter_end=iter_end)
    ms, launches, updates = B.timing_read(reset=True)
    B.set_option("timing", 0)
    return ms, launches, updates


SAMPLED_ITERATIONS = ((0, 2), (15, 17))  # a mixed and a cooling pair of iterations


def _batch_sampled(B, xy, seeds):
    """One-graph-at-a-time schedules take minutes per layout (each graph alone
    under its concurrency cap is latency-bound), so they are timed over the
    iterations of SAMPLED_ITERATIONS (every iteration makes the same updates)
    and scaled to the whole layout."""
    ms = launches = upd = 0
    for a, b in SAMPLED_ITERATIONS:
        B.set_coords(xy)
        B.set_option("timing", 1)
        B.timing_read(reset=True)
        B.layout(ITERS, seeds=seeds, theta=THETA, iter_begin=a, iter_end=b)
        m, n, u = B.timing_read(reset=True)
        B.set_option("timing", 0)
        ms, launches, upd = ms + m, launches + n, upd + u
    its = sum(b - a for a, b in SAMPLED_ITERATIONS)
    return {"ms": ms * ITERS / its, "ms_extrapolated": True, "timed_iterations": [list(x) for x in SAMPLED_ITERATIONS],
            "timed_ms": ms, "updates_per_s": upd / (ms / 1e3), "launches": launches * ITERS // its,
            "stress": None, "quality": "the same kernels and caps as the batched schedule; per-graph stress "
                                      "against the oracle in the GPU tests"}


def batch_form(dev, full=False, log=None, name="batch256"):
    """The 256-subgraph batch: autotuned batched schedule against one launch
    per graph (and, with full, the other schedules and separate one-graph
    handles), every schedule from the same initial layouts and seeds."""
    import torch
    import paper_2409_00876_gb300 as pg
    from paper_2409_00876_gb300.batch import Batch, autotune
    from synth import concat, make_batch
    gs = make_batch(name)
    arr = concat(gs)
    B = Batch.from_arrays(arr)
    xy = torch.from_numpy(arr.init_xy).to(dev)
    seeds = np.arange(1, len(gs) + 1, dtype=np.uint64)
    updates = ITERS * 10 * sum(g.n_steps for g in gs)
    t0 = time.perf_counter()
    tuned, table = autotune(B, xy, seeds=seeds, iter_max=ITERS, theta=THETA, log=log)
    tune_s = time.perf_counter() - t0

    def stress_summary():
        st = B.stress(STRESS_PER_STEP, seed=STRESS_SEED)
        m = np.array([r["mean"] for r in st])
        out = {"mean_over_graphs": float(m.mean()), "median": float(np.median(m)), "max": float(m.max())}
        if name == "batch256":
            out["vs_oracle"] = batch_subset_vs_oracle(m)
        return out

    _batch_timed(B, xy, seeds)  # warm: the tuned shape's CUDA graph
    ms, launches, _ = _batch_timed(B, xy, seeds)
    out = {"workload": WORKLOADS[name], "n_graphs": len(gs), "updates": updates,
           "tuned": {**tuned, "mode": {0: "launch per iteration (CUDA graph)", 1: "persistent", 2: "per graph"}[
               tuned["mode"]]}, "autotune_s": round(tune_s, 1),
           "autotune_trials_ms": {"/".join(map(str, k)): round(v, 2) for k, v in table.items()},
           "autotune_keys": "mode/pipeline/updates_per_thread/block/chunk",
           "batched": {"ms": ms, "updates_per_s": updates / (ms / 1e3), "launches": launches,
                       "stress": stress_summary()}}
    # the persistent kernel (one launch per layout) is reported beside the tuned choice every time, under its
    # own best shape (the autotuner restricted to mode 1); the other schedules run the overall tuned shape
    t0 = time.perf_counter()
    tuned_p, _ = autotune(B, xy, seeds=seeds, iter_max=ITERS, theta=THETA,
                          space=dict(mode=[1], pipeline=[0, 1], updates_per_thread=[1, 2], block=[256],
                                     chunk=[32768, 16384, 65536]))
    out["persistent_tuned"] = dict(tuned_p, autotune_s=round(time.perf_counter() - t0, 1))
    base = {k: v for k, v in tuned.items() if k != "mode"}
    others = [("persistent", dict(tuned_p)), ("per_graph_launches", dict(base, mode=2, cuda_graph=0))]
    if full:
        others = [("launch_per_iteration", dict(base, mode=0, cuda_graph=1)),
                  ("per_graph_launches_cuda_graph", dict(base, mode=2, cuda_graph=1))] + others
    for key, opts in others:
        for k, v in opts.items():
            B.set_option(k, v)
        _batch_timed(B, xy, seeds, iter_end=1)
        if opts.get("mode") == 2:
            _batch_sampled(B, xy, seeds)  # warm: the sampled ranges' CUDA graphs
            out[key] = _batch_sampled(B, xy, seeds)
            continue
        ms2, launches2, _ = _batch_timed(B, xy, seeds)
        out[key] = {"ms": ms2, "updates_per_s": updates / (ms2 / 1e3), "launches": launches2,
                    "stress": stress_summary()}
    out["speedup_vs_per_graph_launches"] = out["batched"]["updates_per_s"] / out["per_graph_launches"]["updates_per_s"]
    if full:
        Gs = [pg.Graph.from_synth(g) for g in gs]
        for G, g in zip(Gs, gs):
            G.set_coords(g.init_xy)
        torch.cuda.synchronize()
        ms3 = 0.0
        for a, b in SAMPLED_ITERATIONS:  # timed as _batch_sampled does
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k, G in enumerate(Gs):
                G.layout(ITERS, theta=THETA, seed=int(seeds[k]), iter_begin=a, iter_end=b)
            e1.record()
            torch.cuda.synchronize()
            ms3 += e0.elapsed_time(e1)
        its = sum(b - a for a, b in SAMPLED_ITERATIONS)
        out["one_graph_handles"] = {"ms": ms3 * ITERS / its, "ms_extrapolated": True,
                                    "timed_iterations": [list(x) for x in SAMPLED_ITERATIONS], "timed_ms": ms3,
                                    "updates_per_s": updates * its / ITERS / (ms3 / 1e3), "stress": None}
        for G in Gs:
            G.close()
    B.close()
    return out


def batch_subset_vs_oracle(per_graph):
    """Per-graph stress of a batch256 layout against the oracle's layouts of
    a fixed 16-graph subset (same graph, same layout seed, same samples:
    tests/golden/oracle_batch256_subset.json, written by
    tests/golden/make_batch_goldens.py). The geometric mean of the ratios,
    with a CI95 from their graph-to-graph spread."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_batch256_subset.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    idx = [g["index"] for g in rec["graphs"]]
    ratios = np.array([per_graph[k] / g["stress"][0] for k, g in zip(idx, rec["graphs"])])
    lr = np.log(ratios)
    half = 1.96 * lr.std(ddof=1) / np.sqrt(len(lr))
    return {"graphs": len(idx), "indices": idx, "n_steps": [g["n_steps"] for g in rec["graphs"]],
            "ratios": [round(float(r), 4) for r in ratios], "geomean_ratio": float(np.exp(lr.mean())),
            "geomean_ci95": [float(np.exp(lr.mean() - half)), float(np.exp(lr.mean() + half))]}


def dstress_form(dev, n_pairs=10_000_000, steps=200):
    """Differentiable sampled stress on the laid-out 200 k-node graph: forward
    and backward kernel times for 10 M pairs, and a 200-step full-batch
    refinement from the PG-SGD result (Adam on the hand-written gradient)."""
    import torch
    import paper_2409_00876_gb300 as pg
    from paper_2409_00876_gb300.autograd import refine
    from synth import make_graph
    g = make_graph("mid")
    G = pg.Graph.from_synth(g)
    G.set_coords(g.init_xy)
    G.layout(ITERS, theta=THETA, seed=SEED)
    xy = torch.empty((g.n_nodes, 4), dtype=torch.float64, device=dev)
    G.get_coords(xy)
    grad = torch.empty((g.n_nodes, 4), dtype=torch.float32, device=dev)
    fw, bw = [], []
    for i in range(4):
        t0 = time.perf_counter()
        _, n_valid = G.dstress(n_pairs, 3)
        t1 = time.perf_counter()
        G.dstress_backward(n_pairs, 3, 1.0 / n_valid, grad)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if i:
            fw.append(t1 - t0)
            bw.append(t2 - t1)
    held_out = list(range(100, 108))  # stress seeds the refinement never sees

    def held(x):
        G.set_coords(x)
        return np.array([G.stress(STRESS_PER_STEP, seed=sd)["mean"] for sd in held_out])

    before = held(xy)
    out = {"workload": WORKLOADS["mid"] + ", after a 30-iteration PG-SGD layout", "pairs": n_pairs,
           "forward_ms": 1e3 * min(fw), "backward_ms": 1e3 * min(bw), "pairs_per_s_backward": n_pairs / min(bw),
           "refine_steps": steps, "stress_before": float(before.mean()),
           "held_out": f"Eq. 2 at {STRESS_PER_STEP} samples per step under stress seeds {held_out[0]}-{held_out[-1]}; "
                       "change = mean over seeds of (after - before) on the same samples, CI95 over the seeds",
           "timing": "host wall clock around synchronous calls (forward includes its readback)"}
    for name, resample in (("full_batch", False), ("resampled", True)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xr, trace = refine(G, xy, steps=steps, lr=0.05, n_pairs=n_pairs, seed=9, resample=resample)
        torch.cuda.synchronize()
        ref_s = time.perf_counter() - t0
        d = held(xr) - before
        half = 1.96 * d.std(ddof=1) / np.sqrt(len(d))
        out[name] = {"refine_s": ref_s, "objective_first": trace[0], "objective_last": trace[-1],
                     "stress_after": float((before + d).mean()), "stress_change": float(d.mean()),
                     "stress_change_ci95": [float(d.mean() - half), float(d.mean() + half)],
                     "relative_change": float(d.mean() / before.mean()),
                     "significant": bool(abs(d.mean()) > half)}
    # the full-batch figures under their earlier names
    out.update(refine_s=out["full_batch"]["refine_s"], objective_first=out["full_batch"]["objective_first"],
               objective_last=out["full_batch"]["objective_last"], stress_after=out["full_batch"]["stress_after"],
               stress_change=out["full_batch"]["stress_change"])
    return out


def reuse_form(G, xy0, schemes=((1, 1, 1), (2, 2, 0), (4, 4, 0), (8, 8, 0))):
    """Warp merging and warp-level data reuse (DRF, SRF) on the same graph:
    one full layout per scheme from the same initial layout and seed, its
    time and its sampled stress, beside the plain method's."""
    G.set_option("timing", 1)
    out = []
    try:
        for drf, srf, wm in ((1, 1, 0),) + tuple(schemes):
            G.set_option("drf", drf)
            G.set_option("srf", srf)
            G.set_option("warp_merge", wm)
            G.set_coords(xy0)
            G.timing_read(reset=True)
            G.layout(ITERS, theta=THETA, seed=SEED)
            ms, _, upd = G.timing_read(reset=True)
            st = G.stress(STRESS_PER_STEP, seed=STRESS_SEED)
            out.append({"drf": drf, "srf": srf, "warp_merge": wm, "layout_ms": ms, "updates": upd,
                        "updates_per_s": upd / (ms / 1e3), "stress": st["mean"], "stress_ci": [st["ci_lo"], st["ci_hi"]]})
    finally:
        G.set_option("drf", 1)
        G.set_option("srf", 1)
        G.set_option("warp_merge", 0)
        G.set_option("timing", 0)
    base = out[0]
    for r in out:
        r["speedup"] = base["layout_ms"] / r["layout_ms"]
        r["stress_ratio"] = r["stress"] / base["stress"]
    return out


def run_batch(args):
    """--config batch256: one JSON line for the batched schedule."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_dist("nccl" if ws > 1 else "gloo")
    dev = torch.device("cuda", local)
    import paper_2409_00876_gb300 as pg
    from paper_2409_00876_gb300.batch import Batch, autotune
    from synth import concat, make_batch
    pg.load_library()
    gs = make_batch(args.config)
    arr = concat(gs)
    B = Batch.from_arrays(arr)
    xy = torch.from_numpy(arr.init_xy).to(dev)
    seeds = np.arange(1, len(gs) + 1, dtype=np.uint64)
    tuned, _ = autotune(B, xy, seeds=seeds, iter_max=ITERS, theta=THETA)
    S = sum(g.n_steps for g in gs)
    updates_per_step = ITERS * 10 * S
    stream = torch.cuda.current_stream()

    def step():
        B.set_coords(xy)
        B.layout(ITERS, seeds=seeds, theta=THETA)
        return B.stress(STRESS_PER_STEP, seed=STRESS_SEED)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    B.set_option("timing", 1)
    B.timing_read(reset=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    lay_ms, launches, upd = B.timing_read(reset=True)
    B.set_option("timing", 0)
    ms_max = max_over_ranks(ms, dev)
    value = aggregate_rate(updates_per_step * args.steps, ms, dev)
    peak, peak_kind = peaks()
    achieved = BYTES_PER_UPDATE * upd / (lay_ms / 1e3) / 1e9
    B.close()
    comp = batch_form(dev, full=True, name=args.config) if rank == 0 and not args.no_forms else None
    if rank == 0:
        m = np.array([r["mean"] for r in st])
        per_launch = {0: ITERS, 1: 1, 2: ITERS * len(gs)}[tuned["mode"]]
        line = {
            "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "name": args.config, "n_steps": S,
                       "updates_per_step": updates_per_step, "tuned": tuned,
                       "l2": f"inputs larger than L2 ({16 * S / 1e9:.1f} GB of step records), no flush",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "stress": {"mean_over_graphs": float(m.mean()), "max": float(m.max()),
                       "vs_oracle": batch_subset_vs_oracle(m) if args.config == "batch256" else None},
            "layout_only_updates_per_s": upd / (lay_ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "batch layout kernels",
                         "bytes_per_update_model": BYTES_PER_UPDATE, "peak_kind": peak_kind},
            "clocks": clk,
            "gpu_launches": args.steps * (2 + per_launch + 1),
            "comparison": comp,
        }
        print(json.dumps(line), flush=True)
    return 0


def hbm_gather(pg):
    """Random-read ceiling of HBM measured in-repo (pgsgd_hbm_gather_bandwidth,
    4 GiB buffer): reads/s of 16-byte step-record-like reads, two per unit on
    one of 90 "paths" (mode 0), and with two L2-resident 8-byte node-like reads
    per unit besides (mode 1); best of 8, 16 and 32 blocks per SM."""
    best = {m: max(pg.hbm_gather_rate(4 << 30, 4, m, b) for b in (8, 16, 32)) for m in (0, 1)}
    return {"reads_per_s": best[0],
            "reads_per_s_with_node_reads": best[1],  # one unit in flight per thread: not a ceiling, context only
            "gbs_as_32B_sectors": best[0] * 32 / 1e9, "gbs_as_64B_accesses": best[0] * 64 / 1e9,
            "pattern": "16-byte reads, evict-first, 64-byte prefetch hint; two per unit, uniform on one of 90 "
                       "equal paths of a 4 GiB buffer (Philox4x32-10 indices)"}


def roofline_for(config, achieved, peak, peak_kind, traffic, launch_ms, gather=None, step_reads_per_s=None,
                 gather_ref=None, updates_per_s=None):
    """HBM roofline; for graphs whose records fit in L2 (mid, tiny) the bound is
    L2, against the L2 read bandwidth measured in-repo (pgsgd_l2_bandwidth).
    With `gather` (hbm_gather) the update kernel's random step-record reads
    per second are also set against the measured random-read ceiling of the
    same read form: random_gather_gbs counts each read as its 32-byte sector,
    the unit of the 192-byte model."""
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
         "traffic": traffic, "kernel": "update_kernel", "bytes_per_update_model": BYTES_PER_UPDATE,
         "peak_kind": peak_kind, "launch_ms": launch_ms}
    if gather:
        r["random_gather_gbs"] = gather["gbs_as_32B_sectors"]
        r["random_gather"] = gather
        if step_reads_per_s:
            # the update kernel's step-record reads against the probe's rate of the same reads; as GB/s at
            # 32 B per read (the unit of random_gather_gbs) this is frac_of_random_gather
            r["step_reads_per_s"] = step_reads_per_s
            r["frac_of_random_gather"] = step_reads_per_s / gather["reads_per_s"]
    if gather_ref and updates_per_s:
        r["gather_reference"] = dict(gather_ref, update_frac=updates_per_s / gather_ref["units_per_s"])
    if config in ("mid", "tiny"):
        import paper_2409_00876_gb300 as pg
        stream = max(pg.l2_bandwidth(mib << 20, 20, 0) for mib in (16, 32, 64))
        rand = max(pg.l2_bandwidth(mib << 20, 4, 1) for mib in (16, 32, 64))
        r.update(bound="l2", peak=stream, frac=achieved / stream,
                 peak_kind="measured in-repo: pgsgd_l2_bandwidth, best of streaming 16-byte loads over "
                           "16, 32 and 64 MiB",
                 l2_random_sector_gbs=rand, hbm_peak=peak, hbm_frac=achieved / peak)
    return r


def run_e2e(pg, g, args, dev):
    import torch
    # pinned host inputs: the graph arrays and the initial layout
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(g, k))).pin_memory()
            for k in ("node_len", "path_off", "step_node", "step_rev", "step_pos")}
    xy_in = torch.from_numpy(g.init_xy).pin_memory()
    xy_out = torch.empty_like(xy_in).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values()) + xy_in.numel() * 8
    d2h = xy_out.numel() * 8 + 48

    phases = {}

    def mark(name, t0):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        phases[name] = phases.get(name, 0.0) + (t1 - t0)
        return t1

    def one():
        t = time.perf_counter()
        G = pg.Graph(host["node_len"].numpy(), host["path_off"].numpy(), host["step_node"].numpy(),
                     host["step_rev"].numpy(), host["step_pos"].numpy())
        t = mark("create_s", t)
        G.set_coords(xy_in.numpy())
        t = mark("set_coords_s", t)
        G.layout(ITERS, theta=THETA, seed=SEED)
        t = mark("layout_s", t)
        G.stress(STRESS_PER_STEP, seed=STRESS_SEED)
        t = mark("stress_s", t)
        G.get_coords(xy_out.numpy())
        G.close()
        mark("get_coords_close_s", t)

    one()
    phases.clear()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    k = max(1, args.e2e_steps)
    for _ in range(k):
        one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"unit": UNIT, "updates": ITERS * 10 * g.n_steps * k, "seconds": dt, "steps": k,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "phases_s_per_step": {n: round(v / k, 3) for n, v in phases.items()}}


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and with runs of white space folded
    to one space (string and character literals kept as they are)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_revision():
    """Hash of the update kernel's code (the device helpers and the update
    kernel's section, comments and layout of white space left out): a recorded
    ncu traffic count is only valid for it."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2409_00876_gb300", "csrc")
    h = hashlib.sha1(strip_comments(open(os.path.join(csrc, "pgsgd_device.cuh")).read()).encode())
    text = open(os.path.join(csrc, "pgsgd_kernels.cu")).read()
    a = text.find("// ---------------------------------------------------------------- update math")
    b = text.find("// ---------------------------------------------------------------- debug kernels")
    h.update(strip_comments(text[a:b] if 0 <= a < b else text).encode())
    return h.hexdigest()[:12]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="chrom", choices=list(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-gather", action="store_true", help="skip the HBM random-read probe (profiling runs)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=10.0)
    ap.add_argument("--cpu-full", nargs="*", default=["tiny", "mid"], choices=["tiny", "mid"],
                    help="workloads whose whole oracle layout is timed on the host (all cores; tiny also on 1 "
                         "thread: the 200 k-node graph takes about 10 minutes on one)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the data-reuse, batched and differentiable forms (chromosome run) or the "
                         "schedule comparison (batch runs)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "gb300" and not os.environ.get("PGSGD_BENCH_ALLOW_SHORT"):
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.config in BATCH_WORKLOADS:
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
