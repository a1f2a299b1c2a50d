#!/usr/bin/env python
"""Benchmark of the CCM hot path on GB300.

Workload (one "step"): the batched parameter sweep over a coupled logistic map
of N=10^4 FP32 points: E=1..10, tau=1..4, 20 library sizes log-spaced 100..9000,
r=250 realizations, both directions (800 cells x 250 x 2 = 4*10^5
realizations, 4.0*10^9 neighbour queries, 8.45*10^12 query-library pairs).
One step = one ccm_run of the whole sweep with the library's defaults (query
order, distance indexing tables for the large-L realizations, library
sampler, one persistent brute-force fused kNN/simplex/rho launch per E for the
rest, one table-scan launch; replayed from a CUDA graph) followed by
ccm_convergence, the per-(pair, E, tau) convergence decision on the rho grid.

Prints one JSON line.  `value` is realizations/s with inputs resident on the
device; `e2e` is the same metric through ccm_run with pinned host buffers
(host->device series copy and device->host rho copy inside the timed region);
`roofline` reports the dominant kernel (the brute-force fused kernels) against
the FP32 ALU peak; `cpu_baseline` is the FP64 oracle on a bounded sample of the
same workload, and `accuracy` checks the GPU's results of that sample against
it (max |d rho|, max relative |d Xhat|, near-tie neighbour swaps);
`brute_force_variant` is the same sweep without tables; `vs_plain_gpu`
compares with the one-launch-per-realization plain GPU CCM on an r=8 subset;
`other_workloads` times the single-job, long-series and network
configurations; `serving` replays the served job stream (2000 jobs, Poisson
arrivals at 0.7 x the calibrated capacity) and reports p50/p99 latency.

Multi-GPU (torchrun): every rank runs its own replica of the sweep (no data
exchange); the barrier and a max-reduction of the timings are the only
collectives.  ``--impl reference`` times the CPU oracle instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CCM realizations/s & neighbour queries/s vs plain GPU CCM; p50/p99 job latency"
UNIT = "realizations/s"
# FP32 peak from unit counts and the maximum clock: 152 SMs x 128 FP32 lanes x
# 2 flops per fused multiply-add x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
KNN_SRC = os.path.join(ROOT, "paper_1905_00565_gb300", "csrc", "knn_fused.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "knn_fused_default_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-units", type=int, default=192,
                    help="realizations in the CPU oracle's sample (also the accuracy check)")
    ap.add_argument("--cpu-pair-budget", type=float, default=3e10,
                    help="stop drawing the sample once its query-library pairs reach this")
    ap.add_argument("--plain-r", type=int, default=8,
                    help="realizations per cell of the plain-comparator subset")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the single-job, long-series and network lines")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-brute", action="store_true",
                    help="skip the brute-force-only (CCM_NO_TABLE) variant")
    ap.add_argument("--serving-jobs", type=int, default=2000)
    ap.add_argument("--scenario", default="", choices=["", "paper"],
                    help="paper: the paper's baseline scenario and its one-at-a-time "
                         "elasticity cases (context, not the bench line)")
    ap.add_argument("--workload", default="sweep", choices=sorted(WORKLOADS),
                    help="sweep (default: the benchmark line), or one of the other "
                         "configurations: single, long, network")
    ap.add_argument("--profile-case", type=int, default=0, metavar="R",
                    help="only run every sweep cell with R realizations through ccm_run "
                         "twice (the small case for ncu captures) and exit")
    return ap.parse_args()


WORKLOADS = {
    "sweep": ("sweep_problem",
              "ccm-sweep: coupled logistic map N=10000 (rx=3.8, ry=3.5, bxy=0.02, byx=0.1), "
              "both directions, E=1..10, tau=1..4, 20 L log-spaced 100..9000, r=250"),
    "single": ("plain_ccm_problem",
               "ccm-single: coupled logistic map N=1000, both directions, E=2, tau=1, "
               "L in {50,100,200,400,800}, r=100"),
    "long": ("long_series_problem",
             "ccm-long: weakly coupled logistic map (byx=0.01, bxy=0) + N(0, 0.01^2) noise, "
             "N=100000, both directions, E=3..6, tau=1, L in {1k,5k,10k,25k,50k}, r=250"),
    "network": ("network_problem",
                "ccm-network: 64-variable coupled logistic network (5% couplings U(0,0.1)), "
                "N=5000, all 4032 ordered pairs, E in {2,3,4}, tau=1, 8 L log-spaced "
                "100..4500, r=250"),
}


def workload_problem(name):
    from paper_1905_00565_gb300 import inputs as I
    return getattr(I, WORKLOADS[name][0])()


def workload_config(name, p):
    return {
        "workload": WORKLOADS[name][1],
        "realizations": p.n_units(),
        "queries": p.queries(),
        "pairs": p.pair_count(),
        "precision": "FP32 distances/selection/weights, FP64 rho moments",
    }


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- multi-rank logic ---
def reduce_max(value: float, dist=None, device=None) -> float:
    """Max over ranks of a per-rank time (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job units per second: every rank runs its own replica, so the job
    processes world x units in the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------ CPU oracle ---
# The CPU-baseline leg: the FP64 oracle (neighbour selection in FP64 too, the
# oracle the accuracy statement names) timed on a bounded, seeded sample of
# the workload's realizations on all host cores; its outputs of that sample
# are kept and, once the GPU has run, the GPU's results of the same
# realizations are checked against them (``accuracy``).
XHAT_FLOOR = 1e-3       # relative-error denominator floor, as a fraction of std(target)
NEAR_TIE = 1e-6         # FP64 (E+1)/(E+2) gap below which a neighbour set may differ


def _oracle_unit(args):
    import oracle
    series, j, i, E, tau, L, k, seed = args
    return oracle.ccm_unit(series, j, i, E, tau, L, k, seed, select_fp64=True, keep=True)


def cpu_sample(p, n_units: int, pair_budget: float, seed: int = 1):
    """A seeded uniform sample of realizations of the workload, cut once its
    query-library pairs reach pair_budget: [(flat index, task)], pairs."""
    import numpy as np
    rng = np.random.default_rng(seed)
    total = p.n_units()
    idx = rng.choice(total, size=min(n_units, total), replace=False)
    shape = (len(p.pairs), len(p.E), len(p.tau), len(p.L), p.r)
    tasks, pairs = [], 0.0
    for flat in idx:
        pi, e, t, l, k = np.unravel_index(int(flat), shape)
        j, i = (int(x) for x in p.pairs[pi])
        E, tau, L = int(p.E[e]), int(p.tau[t]), int(p.L[l])
        tasks.append((int(flat), (p.series, j, i, E, tau, L, int(k), p.seed)))
        pairs += (p.n - (E - 1) * tau) * L
        if pairs >= pair_budget:
            break
    return tasks, pairs


def time_cpu_oracle(p, n_units: int, pair_budget: float, keep: bool = False):
    """The FP64 oracle over a bounded sample on all host cores (spawned workers).
    The rate is scaled to the whole workload by pair count (extrapolated)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    tasks, pairs = cpu_sample(p, n_units, pair_budget)
    cores = os.cpu_count() or 1
    ctxm = mp.get_context("spawn")
    with ctxm.Pool(cores) as pool:
        pool.map(_oracle_unit, [t for _, t in tasks[:cores]])   # warm the workers
        t0 = time.perf_counter()
        outs = pool.map(_oracle_unit, [t for _, t in tasks], chunksize=1)
        dt = time.perf_counter() - t0
    pairs_per_s = pairs / dt
    value = pairs_per_s * p.n_units() / p.pair_count()
    res = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
           "selection": "FP64 (the oracle the accuracy statement names)",
           "sample": f"{len(tasks)} realizations drawn uniformly (seed 1) from the workload, "
                     f"{pairs:.3e} query-library pairs in {dt:.2f} s wall on {cores} "
                     f"processes; rate scaled to the whole workload by pair count",
           "extrapolated": True, "sample_wall_s": dt, "sample_realizations": len(tasks),
           "pairs_per_s": pairs_per_s}
    if keep:
        res["_outputs"] = [(flat, task, out) for (flat, task), out in zip(tasks, outs)]
    return res


def check_accuracy(ccm, ctx, p, rho_sweep, kept):
    """The GPU's results of the CPU leg's sampled realizations against the FP64
    oracle outputs kept there.  Per realization the GPU's library, neighbour
    lists and predictions come from a small run of its (pair, E, tau, L) cell
    with r = k+1 (ccm_run_ex; rho of realization k is bit-identical to the
    sweep's, checked).  Rows whose neighbour sets differ from the FP64 oracle's
    must sit at a near tie (FP64 (E+1)/(E+2) gap below 1e-6 relative); there
    the oracle replays the GPU's sets.  rho is judged against the FP64 oracle,
    or against the replay for a realization with a near-tie swap."""
    import numpy as np
    import oracle
    flat_rho = rho_sweep.reshape(-1)
    worst = {"drho": 0.0, "drho_fp64": 0.0, "dxhat": 0.0}
    ties = units_with_ties = rows = lib_bad = wide_ties = 0
    same_as_sweep = True
    for flat, (series, j, i, E, tau, L, k, seed), (r_o, l_o, n_o, x_o) in kept:
        sub = type(p)(series=series, pairs=np.array([[j, i]], np.int32),
                      E=np.array([E], np.int32), tau=np.array([tau], np.int32),
                      L=np.array([L], np.int64), r=k + 1, seed=seed, name="accuracy")
        plan = ccm.plan_problem(ctx, sub)
        try:
            info = ccm.ccm_plan_get_info(plan)
            rho = np.zeros(ccm.rho_shape(sub))
            lib = np.zeros(info["library_entries"], np.int32)
            nbr = np.zeros(info["neighbour_entries"], np.int32)
            xh = np.zeros(info["n_queries"], np.float32)
            ccm.ccm_run_ex(plan, series, rho, libraries=lib, neighbours=nbr, predictions=xh)
        finally:
            ccm.ccm_plan_destroy(plan)
        n_m = len(x_o)
        l_g = lib[k * L:(k + 1) * L]
        n_g = nbr[k * n_m * (E + 1):(k + 1) * n_m * (E + 1)].reshape(n_m, E + 1)
        x_g = xh[k * n_m:(k + 1) * n_m].astype(np.float64)
        rho_g = float(rho.reshape(-1)[k])
        same_as_sweep &= bool(rho_g == flat_rho[flat] or (np.isnan(rho_g) and np.isnan(flat_rho[flat])))
        lib_bad += int(not np.array_equal(l_g, l_o))
        differ = np.nonzero(np.any(np.sort(n_g, 1) != np.sort(n_o, 1), axis=1))[0]
        if len(differ):
            gap = oracle.query_margin(series[j], E, tau, l_o, differ)
            wide_ties += int(np.sum(gap >= NEAR_TIE))
            ties += len(differ)
            units_with_ties += 1
        den = np.maximum(np.abs(x_o), XHAT_FLOOR * np.std(series[i].astype(np.float64)))
        same = np.ones(n_m, bool)
        same[differ] = False
        dx = float(np.max(np.abs(x_g - x_o)[same] / den[same])) if same.any() else 0.0
        x_rep = oracle.predict(series[j], series[i], E, tau, n_g)
        r_rep = oracle.skill(series[i], E, tau, x_rep)
        dx = max(dx, float(np.max(np.abs(x_g - x_rep) / den)))
        worst["dxhat"] = max(worst["dxhat"], dx)
        if not np.isnan(r_o):
            worst["drho_fp64"] = max(worst["drho_fp64"], abs(rho_g - r_o))
            judged = abs(rho_g - r_rep) if len(differ) else max(abs(rho_g - r_o),
                                                                abs(rho_g - r_rep))
            worst["drho"] = max(worst["drho"], judged)
        rows += n_m
    return {"max_abs_drho": worst["drho"],
            "max_abs_drho_vs_fp64_selection": worst["drho_fp64"],
            "max_rel_dxhat": worst["dxhat"], "near_tie_rows": ties,
            "realizations_with_near_ties": units_with_ties,
            "set_differences_outside_near_ties": wide_ties,
            "libraries_not_bit_exact": lib_bad, "n_checked": len(kept), "rows_checked": rows,
            "sampled_rho_bit_identical_to_sweep": same_as_sweep,
            "tolerances": {"abs_drho": 1e-4, "rel_dxhat": 1e-5, "near_tie_gap": NEAR_TIE},
            "reference": "FP64 oracle (FP64 selection); a realization with a near-tie "
                         "neighbour swap is judged against the oracle's replay of the GPU's "
                         "neighbour sets (max_abs_drho_vs_fp64_selection includes those)"}


# ------------------------------------------------------------ GPU arm ------
def ncu_record():
    """The committed ncu record of the brute-force launches (DRAM bytes per
    sweep, pipe use of the E = 10 launch), if the kernel source still matches
    the profiled one."""
    try:
        rec = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256(open(KNN_SRC, "rb").read()).hexdigest()
    if rec.get("knn_fused_sha256") != h or rec.get("path") != "default":
        return None
    return rec


def search_counts(ccm, ctx, p, dev_flags, s_dev, rho_dev, stream):
    """Work counts of one run of the counting variant (CCM_SEARCH_STATS: same
    results, slower): the query-library pairs the brute-force search began
    (at least the first coordinates) and completed (all E), and the table
    entries the table walks loaded and the queries that missed."""
    plan = ccm.plan_problem(ctx, p, dev_flags | ccm.CCM_SEARCH_STATS)
    try:
        ccm.ccm_run(plan, s_dev, rho_dev, stream=stream)
        stream.synchronize()
        return ccm.ccm_plan_search_stats(plan)
    finally:
        ccm.ccm_plan_destroy(plan)


def time_steps(ccm, plan, s_dev, rho_dev, stream, flush, steps, warmup, after=None):
    """W untimed runs, then K runs each timed by CUDA events on the launching
    stream, with a buffer larger than L2 written before each; returns the
    per-step ms and the per-step stage times."""
    import torch
    for _ in range(warmup):
        ccm.ccm_run(plan, s_dev, rho_dev, stream=stream)
        if after:
            after()
        stream.synchronize()
    step_ms, stage_ms = [], []
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ccm.ccm_run(plan, s_dev, rho_dev, stream=stream)
        if after:
            after()
        e1.record(stream)
        stream.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stage_ms.append(ccm.ccm_plan_stage_times(plan))
    return step_ms, stage_ms


def mean_stages(stage_ms):
    return [sum(x[q] for x in stage_ms) / len(stage_ms) for q in range(4)]


def run_ours(args, rank, world, local_rank, cpu=None):
    import numpy as np
    import torch
    from paper_1905_00565_gb300 import ccm
    from paper_1905_00565_gb300 import inputs as I

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    p = workload_problem(args.workload)
    ctx = ccm.ccm_context_create(local_rank)
    dev_flags = ccm.CCM_INPUT_ON_DEVICE | ccm.CCM_OUTPUT_ON_DEVICE
    plan = ccm.plan_problem(ctx, p, dev_flags)
    info = ccm.ccm_plan_get_info(plan)
    s_dev = torch.from_numpy(p.series).cuda()
    rho_dev = torch.zeros(ccm.rho_shape(p), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    n_rows = len(p.pairs) * len(p.E) * len(p.tau)
    conv_dev = torch.zeros(n_rows * 40, dtype=torch.uint8, device="cuda")
    conv_ms = []

    def convergence():
        em = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        em.record(stream)
        ccm.ccm_convergence(ctx, rho_dev, p.L, out=conv_dev, stream=stream)
        e1.record(stream)
        conv_events.append((em, e1))

    conv_events = []
    # warm-up outside the clock sampling, then the timed steps
    time_steps(ccm, plan, s_dev, rho_dev, stream, flush, 0, args.warmup, convergence)
    conv_events.clear()
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, stage_ms = time_steps(ccm, plan, s_dev, rho_dev, stream, flush, args.steps, 0,
                                   convergence)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    conv_ms = [a.elapsed_time(b) for a, b in conv_events]
    t_step = reduce_max(sum(step_ms) / len(step_ms), dist, "cuda")
    rho_ok = bool(torch.isfinite(rho_dev).all().item())

    # End to end through the public API with pinned host buffers.
    plan_h = ccm.plan_problem(ctx, p, 0)
    s_host = torch.from_numpy(p.series).pin_memory().numpy()
    rho_host = torch.zeros(ccm.rho_shape(p), dtype=torch.float64).pin_memory().numpy()
    ccm.ccm_run(plan_h, s_host, rho_host)
    e2e_s = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        stream.synchronize()
        t0 = time.perf_counter()
        ccm.ccm_run(plan_h, s_host, rho_host)     # H2D, graph, D2H, synchronise
        conv_host = ccm.ccm_convergence(ctx, rho_host, p.L)   # H2D, kernel, D2H
        e2e_s.append(time.perf_counter() - t0)
    e2e_t = reduce_max(sum(e2e_s) / len(e2e_s), dist, "cuda")
    same = bool(np.array_equal(rho_host, rho_dev.cpu().numpy()))
    ccm.ccm_plan_destroy(plan_h)

    out = None
    if rank == 0:
        n_units = info["n_units"]
        st = mean_stages(stage_ms)
        # roofline: the brute-force fused kernels (small-L realizations), the
        # search kernel whose work has a compute roofline (the table scan, the
        # largest stage, is characterised in its own block)
        achieved = info["brute_flop_count"] / (st[2] / 1e3) / 1e12
        ncu_rec = ncu_record() if args.workload == "sweep" else None
        counts = search_counts(ccm, ctx, p, dev_flags, s_dev, rho_dev, stream)
        ex_begun, ex_full = counts["pairs_begun"], counts["pairs_full"]
        idx_bytes = 2 if int(p.series.shape[1]) < 65536 else 4
        out = {
            "metric": METRIC, "value": job_throughput(n_units, world, t_step / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args.workload, p),
                           l2="256 MiB buffer written between timed steps",
                           parallelism="replicas" if world > 1 else "single GPU"),
            "queries_per_s": info["n_queries"] * world / (t_step / 1e3),
            "pairs_per_s": info["pair_count"] * world / (t_step / 1e3),
            "kernel_ms": {"order_and_tables": st[0], "sampler": st[1],
                          "knn_fused_brute_force": st[2], "knn_table_scan": st[3],
                          "convergence": sum(conv_ms) / max(1, len(conv_ms))},
            "neighbour_search": {
                "tables": "distance indexing tables (paper Sect. 3.2), built every step, for "
                          "L >= max(256, sqrt(20 N_m/(E+1)), N_m/40), rows of R entries so that a "
                          "query at the smallest such L misses its E+1 members with probability "
                          "<= 1/(10 L); brute force with exact chunk pruning below",
                "table_bytes": info["table_bytes"],
                "brute_force_share_of_pairs": info["brute_pair_count"] / info["pair_count"],
                "brute_force_share_of_flops": info["brute_flop_count"] / info["flop_count"],
                "table_query_share": info["table_query_count"] / max(1, info["search_query_count"])},
            # the table-scan kernel: the largest stage, but a lookup walk with no
            # flop or byte count of the exhaustive method to put against a peak
            "table_scan": {
                "kernel": "knn_table_kernel<E>, one launch per E per step: each query walks "
                          "its table row until every realization of its group (up to 4 of a "
                          "cell) has E+1 library members, then the simplex/moment epilogue",
                "share_of_step": st[3] / t_step,
                "query_realizations_per_s": info["table_query_count"] / (st[3] / 1e3),
                # from the counting run: rank entries the walks loaded (one walk
                # serves up to four realizations) and the index bytes they read
                "entries_loaded_per_s": counts["table_entries"] / (st[3] / 1e3),
                "index_bytes_per_s": counts["table_entries"] * idx_bytes / (st[3] / 1e3),
                "library_scan_fallbacks": counts["table_fallbacks"],
                "brute_force_query_realizations_per_s":
                    (info["search_query_count"] - info["table_query_count"]) / (st[2] / 1e3),
                "bound": "issue and L2 latency (see the committed ncu summary)"},
            "convergence": {"rows": n_rows, "converged_rows": int(conv_host["converged"].sum()),
                            "test": f"one-sided Jonckheere-Terpstra over the {len(p.L)} L "
                                    "groups, z > 1.645"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                         # the committed capture covers the sweep workload only
                         "traffic": (ncu_rec or {}).get("dram_bytes_per_full_sweep"),
                         "traffic_unit": "DRAM bytes per step, all brute-force launches "
                                         "(ncu, scaled from an r=8 capture)",
                         "algorithmic_bytes": "4L per realization (library indices) + 8 (rho)",
                         "kernel": "knn_fused_kernel<E> (brute force), one launch per E per step "
                                   "over the realizations below the table threshold; 3E FP32 "
                                   "flops per query-library pair of those realizations (the "
                                   "method's exhaustive work, including the pairs that exact "
                                   "chunk pruning skips)",
                         "brute_pairs_per_s": info["brute_pair_count"] / (st[2] / 1e3),
                         # pairs the search evaluated (pruning skips the rest), counted
                         # by a separate run of the counting variant, per second of the
                         # timed brute-force stage
                         "executed_pairs_per_s": ex_begun / (st[2] / 1e3),
                         "completed_pairs_per_s": ex_full / (st[2] / 1e3),
                         "ncu_e10_launch": (ncu_rec or {}).get("pipes_e10"),
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
            "e2e": {"value": job_throughput(n_units, world, e2e_t), "unit": UNIT,
                    "h2d_bytes_per_step": int(p.series.nbytes) + int(rho_host.nbytes),
                    "d2h_bytes_per_step": int(rho_host.nbytes) + int(conv_host.nbytes),
                    "ms_per_step": e2e_t * 1e3, "same_rho_as_device_path": same},
            # per step: query order, tables, sampler, brute force per E, table scan,
            # convergence
            "gpu_launches": (info["launches_per_run"] + 1) * args.steps,
            "clocks": clk,
            "rho_finite": rho_ok,
        }
        if cpu is not None and "_outputs" in cpu:
            out["accuracy"] = check_accuracy(ccm, ctx, p, rho_dev.cpu().numpy(),
                                             cpu.pop("_outputs"))
        extras = world == 1   # a multi-rank run times the replicas only
        if extras and not args.no_brute:
            bv = brute_variant(ccm, ctx, p, torch, min(args.steps, 3), 1, rho_dev, flush, stream)
            bv["default_speedup"] = out["value"] / bv["value"]
            out["brute_force_variant"] = bv
        if extras and not args.no_plain:
            out["vs_plain_gpu"] = compare_plain(ccm, ctx, I, p, torch, args.plain_r)
        if extras and not args.no_other and args.workload == "sweep":
            out["other_workloads"] = other_workloads(ccm, ctx, torch, stream, flush, args)
        if extras and not args.no_serving:
            out["serving"] = serve_stream(ccm, I, args.serving_jobs, local_rank)
    ccm.ccm_plan_destroy(plan)
    ccm.ccm_context_destroy(ctx)
    return out


def other_workloads(ccm, ctx, torch, stream, flush, args):
    """The single-job, long-series and network configurations, each timed like
    the main line (device-resident inputs, CUDA events, L2 flushed between
    steps), a few steps each."""
    res = {}
    flags = ccm.CCM_INPUT_ON_DEVICE | ccm.CCM_OUTPUT_ON_DEVICE
    steps = max(1, min(args.steps, 5))
    for name in ("single", "long", "network"):
        p = workload_problem(name)
        plan = ccm.plan_problem(ctx, p, flags)
        try:
            info = ccm.ccm_plan_get_info(plan)
            s_dev = torch.from_numpy(p.series).cuda()
            rho = torch.zeros(ccm.rho_shape(p), dtype=torch.float64, device="cuda")
            step_ms, stage_ms = time_steps(ccm, plan, s_dev, rho, stream, flush, steps, 2)
            t = sum(step_ms) / len(step_ms)
            st = mean_stages(stage_ms)
            res[name] = {"value": info["n_units"] / (t / 1e3), "unit": UNIT, "ms_per_step": t,
                         "steps": steps, "warmup": 2,
                         "queries_per_s": info["n_queries"] / (t / 1e3),
                         "kernel_ms": {"order_and_tables": st[0], "sampler": st[1],
                                       "knn_fused_brute_force": st[2], "knn_table_scan": st[3]},
                         "rho_finite": bool(torch.isfinite(rho).all().item()),
                         "config": workload_config(name, p)}
            del s_dev, rho
        finally:
            ccm.ccm_plan_destroy(plan)
    return res


def serve_stream(ccm, I, n_jobs: int, device: int):
    """Served request stream: the first n_jobs of the seeded job stream (lengths
    log-uniform 500..50000, E 1..10, tau 1..5, r in {100, 250}; all 2000 by
    default).  Capacity is calibrated by submitting every job at once; the
    stream is then replayed with Poisson arrivals at 0.7 x that capacity, and
    per-job latency (submit to finish, on the library's clock) is reported."""
    import numpy as np
    jobs = I.job_stream(n_jobs=n_jobs, rate_per_s=1.0)
    ctx = ccm.ccm_context_create(device)

    def run(arrivals):
        t0 = time.perf_counter()
        tickets = []
        for a, j in zip(arrivals, jobs):
            delay = a - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            q = j.problem
            tickets.append(ccm.ccm_submit(ctx, q.series, q.pairs, q.E, q.tau, q.L, q.r, q.seed))
        lat, first, last = [], None, None
        for t, j in zip(tickets, jobs):
            while True:
                st, sub, start, fin = ccm.ccm_job_times(ctx, t)
                if st == ccm.CCM_OK:
                    break
                time.sleep(0.001)
            rho = np.zeros(ccm.rho_shape(j.problem))
            ccm.ccm_poll(ctx, t, rho, 0)
            lat.append(fin - sub)
            first = sub if first is None else min(first, sub)
            last = fin if last is None else max(last, fin)
        return np.array(lat), last - first

    try:
        _, span = run([0.0] * n_jobs)                  # calibration: all at once
        capacity = n_jobs / span
        rate = 0.7 * capacity
        arrivals = [j.arrival_s / rate for j in jobs]  # unit-rate Poisson times rescaled
        lat, span2 = run(arrivals)
    finally:
        ccm.ccm_context_destroy(ctx)
    units = sum(j.problem.n_units() for j in jobs)
    pairs = sum(j.problem.pair_count() for j in jobs)
    return {"jobs": n_jobs,
            "stream": f"the first {n_jobs} jobs of the seeded served stream (seed 20190505)",
            "capacity_jobs_per_s": capacity, "arrival_rate_per_s": rate,
            "calibration": f"all {n_jobs} jobs submitted at once: {span:.2f} s",
            "p50_latency_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_latency_ms": float(np.percentile(lat, 99) * 1e3),
            "max_latency_ms": float(lat.max() * 1e3),
            "realizations_per_s": units / span2, "realizations": units, "pairs": float(pairs),
            "makespan_s": span2}


def brute_variant(ccm, ctx, p, torch, steps: int, warmup: int, rho_ref, flush, stream):
    """The same sweep with CCM_NO_TABLE: every realization searched by the
    brute-force fused kernels (with exact chunk pruning); bit-identical rho."""
    flags = ccm.CCM_INPUT_ON_DEVICE | ccm.CCM_OUTPUT_ON_DEVICE | ccm.CCM_NO_TABLE
    plan = ccm.plan_problem(ctx, p, flags)
    info = ccm.ccm_plan_get_info(plan)
    s_dev = torch.from_numpy(p.series).cuda()
    rho = torch.zeros(ccm.rho_shape(p), dtype=torch.float64, device="cuda")
    step_ms, stages = time_steps(ccm, plan, s_dev, rho, stream, flush, steps, max(1, warmup))
    same = bool(torch.equal(rho, rho_ref))
    ccm.ccm_plan_destroy(plan)
    t = sum(step_ms) / len(step_ms)
    st = mean_stages(stages)
    achieved = info["flop_count"] / (st[2] / 1e3) / 1e12
    return {"value": info["n_units"] / (t / 1e3), "unit": UNIT, "ms_per_step": t,
            "steps": steps,
            "stage_ms": {"order": st[0], "sampler": st[1], "knn_fused_brute_force": st[2]},
            "roofline_frac": achieved / FP32_PEAK_TFLOPS, "achieved_tflops": achieved,
            "same_rho_bits_as_default": same}


def compare_plain(ccm, ctx, I, p, torch, r: int):
    """Fused sweep vs the plain one-launch-per-realization CCM on the same subset:
    every cell of the workload with r realizations."""
    sub = I.subproblem(p, r=r)
    flags = ccm.CCM_INPUT_ON_DEVICE | ccm.CCM_OUTPUT_ON_DEVICE
    plan = ccm.plan_problem(ctx, sub, flags)
    s = torch.from_numpy(sub.series).cuda()
    ra = torch.zeros(ccm.rho_shape(sub), dtype=torch.float64, device="cuda")
    rb = torch.zeros_like(ra)
    st = torch.cuda.Stream()
    ccm.ccm_run(plan, s, ra, stream=st)
    ccm.ccm_run_plain(plan, s, rb, stream=st)
    st.synchronize()
    t0 = time.perf_counter()
    ccm.ccm_run(plan, s, ra, stream=st)
    st.synchronize()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    ccm.ccm_run_plain(plan, s, rb, stream=st)
    st.synchronize()
    tp = time.perf_counter() - t0
    ccm.ccm_plan_destroy(plan)
    n = sub.n_units()
    return {"subset": f"every (pair, E, tau, L) cell of the workload with r={r} "
                      f"({n} realizations)",
            "fused_realizations_per_s": n / tf, "plain_realizations_per_s": n / tp,
            "speedup": tp / tf,
            "max_abs_rho_diff": float((ra - rb).abs().max().item())}


def profile_case(r: int):
    """Every sweep cell with r realizations, ccm_run twice (graph path)."""
    import numpy as np
    from paper_1905_00565_gb300 import ccm
    from paper_1905_00565_gb300 import inputs as I
    p = I.subproblem(I.sweep_problem(), r=r)
    ctx = ccm.ccm_context_create(0)
    plan = ccm.plan_problem(ctx, p)
    rho = np.zeros(ccm.rho_shape(p))
    for _ in range(2):
        ccm.ccm_run(plan, p.series, rho)
    print(json.dumps({"profile_case_r": r, "realizations": p.n_units(),
                      "kernel_ms": ccm.ccm_plan_kernel_times(plan),
                      "flops": ccm.ccm_plan_get_info(plan)["flop_count"]}))
    ccm.ccm_plan_destroy(plan)
    ccm.ccm_context_destroy(ctx)


def paper_scenario(args):
    """The paper's baseline scenario (N=4000, r=500, L in {500,1000,2000}, E and
    tau in {1,2,4}) and its elasticity cases (one of L, E, tau fixed to each of
    its three values, the others as in the baseline), on the GPU with brute
    force and with distance indexing tables, and on one host core with the
    oracle (a seeded sample of 2 realizations per cell, scaled to r=500).
    Prints one JSON line of times and doubling ratios; the paper's ratios
    (Spark, unnamed series) are quoted beside them as context."""
    import numpy as np
    import torch
    import oracle
    from paper_1905_00565_gb300 import ccm
    from paper_1905_00565_gb300 import inputs as I

    base = I.paper_scenario_problem()
    cases = {"baseline": base}
    for axis in ("L", "E", "tau"):
        for q in range(3):
            cases[f"{axis}={int(getattr(base, axis)[q])}"] = I.subproblem(base, **{axis: [q]})
    ctx = ccm.ccm_context_create(0)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    s_dev = torch.from_numpy(base.series).cuda()
    dev = ccm.CCM_INPUT_ON_DEVICE | ccm.CCM_OUTPUT_ON_DEVICE
    res = {}
    for name, p in cases.items():
        row = {"realizations": p.n_units()}
        for label, flags in (("gpu_ms", dev | ccm.CCM_NO_TABLE), ("gpu_table_ms", dev)):
            plan = ccm.plan_problem(ctx, p, flags)
            rho = torch.zeros(ccm.rho_shape(p), dtype=torch.float64, device="cuda")
            for _ in range(max(3, args.warmup)):
                ccm.ccm_run(plan, s_dev, rho, stream=stream)
            ts = []
            for k in range(max(5, args.steps)):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 0xFF)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ccm.ccm_run(plan, s_dev, rho, stream=stream)
                e1.record(stream)
                stream.synchronize()
                ts.append(e0.elapsed_time(e1))
            row[label] = statistics.median(ts)
            ccm.ccm_plan_destroy(plan)
        sub = I.subproblem(p, r=2)
        t0 = time.perf_counter()
        oracle.ccm(sub.series, sub.pairs, sub.E, sub.tau, sub.L, sub.r, sub.seed)
        row["oracle_1core_s"] = (time.perf_counter() - t0) * p.r / sub.r
        res[name] = row
    ccm.ccm_context_destroy(ctx)

    def ratios(axis, key):
        vals = [res[f"{axis}={int(v)}"][key] for v in getattr(base, axis)]
        return [vals[1] / vals[0], vals[2] / vals[1]]

    out = {"scenario": "paper baseline and elasticity (Table 2) on a synthetic stand-in",
           "workload": "coupled logistic map N=4000, both directions, r=500, "
                       "L in {500,1000,2000}, E and tau in {1,2,4}",
           "cases": res,
           "doubling_ratios": {f"{axis}": {k: ratios(axis, k) for k in
                                           ("gpu_ms", "gpu_table_ms", "oracle_1core_s")}
                               for axis in ("L", "E", "tau")},
           "paper_context": {"L_doubling_single_threaded": 4.06, "L_doubling_parallel": 1.11,
                             "tau_doubling_single_threaded": 1.13,
                             "E_or_tau_doubling_parallel": "almost no impact",
                             "hardware": "Spark on YARN, 1 master + 5 workers, 4 cores each"}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.workload in ("long", "network"):
        # the plain comparator would take minutes here; the served stream is the
        # same for every workload
        args.no_plain = args.no_serving = True
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.scenario == "paper":
        paper_scenario(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        p = workload_problem(args.workload)
        for _ in range(args.warmup):
            time_cpu_oracle(p, 16, args.cpu_pair_budget / 8)
        vals = [time_cpu_oracle(p, args.cpu_sample_units, args.cpu_pair_budget)
                for _ in range(args.steps)]
        v = statistics.mean(x["value"] for x in vals)
        wall_ms = 1e3 * statistics.mean(x["sample_wall_s"] for x in vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
                # one step is one bounded sample of the workload, timed; the value
                # is that sample's pair rate scaled to the whole workload
                "ms_per_step": wall_ms, "extrapolated": True,
                "step": f"{vals[-1]['sample_realizations']} sampled realizations of the "
                        "workload (FP64 oracle on all host cores)",
                "extrapolated_ms_per_full_workload": 1e3 * p.n_units() / v,
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(workload_config(args.workload, p),
                               l2="not applicable (host cores)", parallelism="host processes"),
                "cpu_baseline": dict(vals[-1], value=v),
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    # the CPU baseline runs before any GPU work so that its spawned workers start clean
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = time_cpu_oracle(workload_problem(args.workload), args.cpu_sample_units,
                              args.cpu_pair_budget, keep=True)
    out = run_ours(args, rank, world, local_rank, cpu)
    if rank == 0:
        out["cpu_baseline"] = cpu
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
