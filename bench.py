"""Throughput of the AIDW hot path (grid build + grid kNN + all-points
weighting) on GB300, printed as one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--scaling weak|strong] [--configs all|none]

A step is one pass of the whole path over one batch: build the even grid of
the data points, find every query's k nearest neighbours, compute alpha and
the weighted prediction of Eq. 1 over all data points.  The headline
workload is n = m = 1,048,576 points uniform in [0,1000]^2, k = 10, float32
with compensated sums (AIDW_FP32_COMP).  On one GPU the line also carries a
``configs`` record with every other workload measured in the same run
(clustered data at k = 10 and 20, the 4M precision form against the float64
GPU path, the 512-job batch, the paper's size sweep), each with its own
step time, roofline fraction and error against the oracle.

Under torchrun (N > 1) every rank builds its own grid from the same data.
``--scaling weak`` (default): every rank interpolates its own seeded query
set of the full size.  ``--scaling strong``: the one query set is split
into N contiguous slices (``aidw_interpolate_shard``).  Nothing is
exchanged on the data path; rank 0 prints the queries of all ranks divided
by the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle (the only reference this
method has) on the host cores, each step a bounded sample of the queries.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AIDW interpolated points/s at n=m=1M (kNN+weighting), FP32-comp vs FP64 plain"
UNIT = "points/s"
L2_FLUSH_BYTES = 256 << 20
# Warp instructions each SM can issue per clock (4 schedulers, one warp of 32
# threads each): the issue ceiling of the weighting loop, in thread
# instructions per SM per clock.
SM_ISSUE_LANES_PER_CLK = 128.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=1 << 20, help="data points = queries")
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--workload", choices=("uniform", "clustered", "batch"), default="uniform")
    ap.add_argument("--scaling", choices=("weak", "strong"), default="weak",
                    help="N > 1: every rank its own full query set (weak) or one slice of "
                         "one query set (strong)")
    ap.add_argument("--jobs", type=int, default=512, help="jobs of the batch workload")
    ap.add_argument("--no-tune", action="store_true", help="batch: skip the autotuner")
    ap.add_argument("--cell-scale", type=float, default=0.0,
                    help="grid cell width / r_exp (<= 0: the library's choice)")
    ap.add_argument("--mode", choices=("aidw", "local", "knn", "knn-table", "sweep", "knn-rule"),
                    default="aidw",
                    help="aidw: Eq. 1 over all points; local: Eq. 1 over the k nearest; "
                         "knn-table: grid vs all-points kNN at the paper's sizes; "
                         "sweep: the full step at the paper's sizes")
    ap.add_argument("--configs", choices=("all", "none"), default="all",
                    help="one GPU, headline workload: also measure the other workloads")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-queries", type=int, default=16384)
    ap.add_argument("--precision-fp64-queries", type=int, default=65536,
                    help="4M precision form: queries the float64 GPU path runs on")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(seconds: float, device=None) -> float:
    """The slowest rank's time (all ranks call it; no-op on one rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cores() -> int:
    """Cores this process may run on; the oracle legs use all of them (a
    launcher may set OMP_NUM_THREADS=1 per rank, which they override)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def whole_job_value(world: int, units_per_rank: int, steps: int, seconds: float) -> float:
    """Units processed by all ranks over the timed steps, per second of the
    slowest rank (weak scaling: every rank has the same amount of work)."""
    return world * units_per_rank * steps / seconds


def strong_value(total_units: int, steps: int, seconds: float) -> float:
    """Strong scaling: the ranks share one set of total_units per step."""
    return total_units * steps / seconds


def make_workload(args, rank, scaling: str = "weak"):
    from paper_1601_05904_gb300 import inputs
    if args.workload == "uniform":
        w = inputs.uniform_kilo(n=args.n, k=args.k, seed=1)
    else:
        w = inputs.clustered_kilo(n=args.n, k=args.k, seed=2)
    if rank and scaling == "weak":
        # each rank its own queries over the same data (weak scaling)
        rng = np.random.default_rng(10_000 + rank)
        w.qx, w.qy = inputs.uniform_points(rng, w.m, 0.0, inputs.SIDE_KILO)
    return w


def workload_config(args, world, precision=None, scaling="weak"):
    if world > 1:
        par = (f"query-sharded x{world}: one query set split into contiguous slices"
               if scaling == "strong" else f"query-sharded x{world}: a query set per rank")
    else:
        par = "single GPU"
    return {"workload": f"{args.workload} n=m={args.n} in [0,1000]^2, k={args.k}, "
                        "alpha levels 1..5, R_min/R_max 0/2",
            "n_data": args.n,
            "n_query_per_gpu": (args.n if scaling == "weak" else -(-args.n // world)), "k": args.k,
            "precision": precision or "FP32-comp (SFU exp2/log2, TwoSum-compensated f32 "
                                      "sums, f64 final divide; alpha in f32 with a "
                                      "compensated r_obs sum)",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "parallelism": par}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[4 + i].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows),
                   power_w_max=max((num(r[2]) or 0.0) for r in rows))
        return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


# ---- roofline accounting ---------------------------------------------------------

def _pipe_times(rates, mix, xe, xl, overhead):
    """SM clocks per pair on each limiting resource when a share xe of the
    exp2s and xl of the log2s run as FMA-pipe polynomials."""
    la, ia = mix["fma_lanes"], mix["instr"]
    sfu = (1.0 - xl) / rates["lg2"] + (1.0 - xe) / rates["ex2"]
    fma = (la["base"] + xe * la["exp2_poly"] + xl * la["lg2_poly"]) / rates["ffma2_lanes"]
    issue = (ia["base"] + (1.0 - xl) + (1.0 - xe) + xe * ia["exp2_poly"] + xl * ia["lg2_poly"]
             + overhead) / SM_ISSUE_LANES_PER_CLK
    return {"sfu": sfu, "fma": fma, "issue": issue}


def weight_pair_bounds(rates, mix, overhead: float = 0.0):
    """Pair-rate ceilings (pairs per SM per clock) of the float32 weighting
    loop from the measured pipe rates and the loop's counted work per pair:

    sfu_both  both transcendentals on the SFU (1 / (1/r_lg2 + 1/r_ex2));
    own_mix   the kernel as launched: the slowest of SFU, FMA pipe and issue
              for its split of exp2/log2 between SFU and FMA-pipe polynomials;
    joint     the best split of both over [0, 1] (steps of 1/64) under the
              same three limits: no split of this loop can beat it."""
    xe = mix["poly_exp2"] / mix["products"]
    xl = mix["poly_lg2"] / mix["products"]
    own = _pipe_times(rates, mix, xe, xl, overhead)
    lim = max(own, key=own.get)
    best = None
    for a in range(65):
        for b in range(65):
            t = _pipe_times(rates, mix, a / 64.0, b / 64.0, overhead)
            r = 1.0 / max(t.values())
            if best is None or r > best[0]:
                best = (r, a / 64.0, b / 64.0, max(t, key=t.get))
    return {"sfu_both": 1.0 / (1.0 / rates["lg2"] + 1.0 / rates["ex2"]),
            "own_mix": 1.0 / own[lim], "own_mix_limit": lim,
            "own_mix_per_resource": {k: 1.0 / v for k, v in own.items()},
            "joint": best[0], "joint_split": {"exp2_on_fma": best[1], "lg2_on_fma": best[2]},
            "joint_limit": best[3], "split": {"exp2_on_fma": xe, "lg2_on_fma": xl}}


def weight_roofline(pairs_per_launch, ms_per_launch, rates, mix, sms, mhz, traffic=None,
                    loop=None):
    """Roofline record of the float32 weighting kernel (Gpair/s).  `peak` is
    the kernel's own-mix ceiling; the line also states the fraction of the
    best-split ceiling and of the both-on-SFU ceiling, and (loop) the rate
    of the kernel's inner loop run alone (aidw_probe_weight_loop) beside the
    kernel's own rate per SM per clock."""
    b = weight_pair_bounds(rates, mix)
    scale = sms * mhz * 1e6 / 1e9
    achieved = pairs_per_launch / (ms_per_launch / 1000.0) / 1e9 if ms_per_launch else None
    peak = b["own_mix"] * scale

    def frac(p):
        return achieved / p if achieved else None
    replica = None
    if loop and achieved:
        per_clk = achieved / scale
        replica = {"kernel_pairs_per_sm_clk": per_clk,
                   "loop_alone_pairs_per_sm_clk": loop,
                   "kernel_over_loop_alone": {c: (per_clk / r if r else None)
                                              for c, r in loop.items()},
                   "basis": "aidw_probe_weight_loop: the kernel's compiled inner loop over a "
                            "shared-memory tile filled once (no copies, waits or barriers), "
                            "at 2 CTAs per SM (the kernel's 128-register form) and 3 (an "
                            "80-register form), clock64-timed; the kernel's rate at the "
                            f"{mhz:.0f} MHz of the roofline"}
    return {"bound": "alu", "kernel": "k_weight_f32 (all-points weighting, Eq. 1)",
            "achieved": achieved, "peak": peak, "unit": "Gpair/s", "frac": frac(peak),
            "peak_joint": b["joint"] * scale, "frac_joint": frac(b["joint"] * scale),
            "peak_sfu_both": b["sfu_both"] * scale, "frac_sfu_both": frac(b["sfu_both"] * scale),
            "traffic": traffic,
            "peak_basis": (f"own mix: {b['split']['exp2_on_fma']:.3f} of exp2 and "
                           f"{b['split']['lg2_on_fma']:.3f} of log2 on FMA-pipe polynomials, "
                           f"limit {b['own_mix_limit']} = {b['own_mix']:.2f} pairs per SM per "
                           f"clock (measured lg2 {rates['lg2']:.2f}, ex2 {rates['ex2']:.2f}, "
                           f"packed FMA {rates['ffma2_lanes']:.1f} lanes per SM per clock; "
                           f"issue {SM_ISSUE_LANES_PER_CLK:.0f}) x {sms} SMs x {mhz:.0f} MHz; "
                           f"joint: best split (exp2 {b['joint_split']['exp2_on_fma']:.3f}, "
                           f"log2 {b['joint_split']['lg2_on_fma']:.3f}) = {b['joint']:.2f} "
                           f"limited by {b['joint_limit']}; sfu_both = {b['sfu_both']:.2f}"),
            "pipe_rates_per_sm_clk": rates, "mix": mix, "loop_alone": replica}


# Algorithmic DRAM bytes of the two memory-side stages (compulsory traffic:
# every input read once, every output written once; intermediates of the
# implementation are not counted).
GRID_BYTES_PER_POINT = 12 + 16 + 12 + 4   # x, y, z in; Point, weighting tile, perm out
GRID_BYTES_PER_CELL = 4                   # cell heads out
KNN_BYTES_PER_QUERY = 8 + 24              # qx, qy in; kNN record out (alpha, hit z, d1^2, hits)
KNN_BYTES_PER_POINT = 16                  # cell-ordered points read once
KNN_BYTES_PER_CELL = 4                    # cell heads read once


def stage_rooflines(stage, n_data, n_query, n_cells, hbm_gbs):
    """HBM roofline records of the grid build and the kNN stage of one step,
    from the library's stage events: stage = {name: (ms, launches)} per step
    (one grid build and one kNN call per step)."""
    out = {}
    g_ms, g_l = stage.get("grid_build", (0.0, 0))
    k_ms, k_l = stage.get("knn", (0.0, 0))
    if g_ms > 0:
        by = GRID_BYTES_PER_POINT * n_data + GRID_BYTES_PER_CELL * (n_cells + 1)
        ach = by / (g_ms / 1000.0) / 1e9
        out["grid_build"] = {"bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
                             "frac": ach / hbm_gbs, "ms": g_ms, "algorithmic_bytes": by,
                             "launches": g_l,
                             "note": "launch- and latency-bound: a chain of small kernels "
                                     "(bounding box and dimensions, keys, scan, scatter, "
                                     "fix-up)"}
    if k_ms > 0:
        by = KNN_BYTES_PER_QUERY * n_query + KNN_BYTES_PER_POINT * n_data + \
            KNN_BYTES_PER_CELL * (n_cells + 1)
        ach = by / (k_ms / 1000.0) / 1e9
        out["knn"] = {"bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
                      "frac": ach / hbm_gbs, "ms": k_ms, "algorithmic_bytes": by,
                      "launches": k_l,
                      "note": "bound by the SM, not by memory: one thread per query "
                              "walks its own cells and sorts its own candidates, so a "
                              "warp instruction runs on 11.7 of 32 lanes on average; ncu "
                              "at 1M: issue 58 % active, ALU pipe 66 % (top-k compares "
                              "and selects), 4 % of L2 and 1 % of DRAM throughput"}
    return out


# ---- oracle legs -------------------------------------------------------------------

def _oracle_sample(w, seconds: float, seed: int, local: bool = False, pool=None):
    """The oracle on a query sample sized to about `seconds` on all host
    cores.  Returns (sample indices, oracle results, seconds, cores)."""
    import oracle
    from paper_1601_05904_gb300 import inputs
    oracle.build()
    fn = oracle.aidw_local if local else oracle.aidw
    cores = host_cores() if oracle.has_openmp() else 1
    idx = np.arange(w.m) if pool is None else np.asarray(pool)
    probe = max(cores, 8)
    s = idx[inputs.query_subsample(idx.size, probe, seed=seed)]
    t0 = time.perf_counter()
    fn(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k, nthreads=cores)
    per_q = (time.perf_counter() - t0) / probe
    count = int(max(probe, min(idx.size, seconds / max(per_q, 1e-9))))
    s = idx[inputs.query_subsample(idx.size, count, seed=seed + 1)]
    t0 = time.perf_counter()
    ref = fn(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k, nthreads=cores)
    return s, ref, time.perf_counter() - t0, cores


def cpu_baseline(w, seconds: float, rank: int, local: bool = False):
    """The oracle as it stands, on the host cores, over a bounded query sample.
    Returns (baseline dict, sample indices, oracle results on the sample)."""
    s, ref, dt, cores = _oracle_sample(w, seconds, 2024 + rank, local)
    return ({"value": s.size / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"{s.size} of {w.m} queries against all {w.n} data points "
                       f"({dt:.1f} s, FP64, brute-force kNN with full sort)"}, s, ref)


def error_figures(z_test, z_ref, scale):
    """Z17's two error figures: max / mean |z - z_ref| / S_q, and the plain
    relative error |z - z_ref| / |z_ref| on queries with |z_ref| >= 0.1 S_q."""
    z_test = np.asarray(z_test, np.float64)
    z_ref = np.asarray(z_ref, np.float64)
    scale = np.asarray(scale, np.float64)
    e = np.abs(z_test - z_ref) / np.maximum(scale, np.finfo(np.float64).tiny)
    big = np.abs(z_ref) >= 0.1 * scale
    rel = np.abs(z_test[big] - z_ref[big]) / np.abs(z_ref[big]) if big.any() else np.zeros(1)
    return {"max_norm_err": float(e.max()), "mean_norm_err": float(e.mean()),
            "max_rel_err_large": float(rel.max()), "large_queries": int(big.sum())}


ERROR_MEASURE = ("norm: max_q |z - z_ref| / S_q with S_q = sum w|z| / sum w; "
                 "rel_large: |z - z_ref| / |z_ref| over queries with |z_ref| >= 0.1 S_q")


def accuracy_on_sample(binding, pkg, t, w, s, ref, params, local, z32_all):
    """Error of the GPU predictions against the oracle on a query sample:
    the FP32-comp output of the timed steps and the FP64 path run on the
    same queries, and the largest alpha difference."""
    import torch
    interp = binding.aidw_interpolate_local if local else binding.aidw_interpolate
    idx = torch.from_numpy(s).to(t["qx"].device)
    qx, qy = t["qx"][idx].contiguous(), t["qy"][idx].contiguous()
    g = binding.aidw_grid_build(t["x"], t["y"], t["z"], params)
    _, a32 = interp(g, qx, qy, params, want_alpha=True)
    p64 = pkg.Params(k=params.k, precision=binding.AIDW_FP64_PLAIN)
    z64, _ = interp(g, qx, qy, p64)
    torch.cuda.synchronize()
    g.destroy()
    f32 = error_figures(z32_all[s], ref["z"], ref["scale"])
    f64 = error_figures(z64.cpu().numpy(), ref["z"], ref["scale"])
    ea = np.abs(a32.cpu().numpy().astype(np.float64) - ref["alpha"])
    return {"queries": int(s.size), "fp32_comp_max_norm_err": f32["max_norm_err"],
            "fp32_comp_mean_norm_err": f32["mean_norm_err"],
            "fp32_comp_max_rel_err_large": f32["max_rel_err_large"],
            "fp64_max_norm_err": f64["max_norm_err"],
            "fp64_max_rel_err_large": f64["max_rel_err_large"],
            "large_queries": f32["large_queries"],
            "alpha_max_abs_err": float(ea.max()),
            "tolerance": {"fp32_comp": 1e-5, "fp64": 1e-9}, "measure": ERROR_MEASURE}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args, 0)
    import oracle
    from paper_1601_05904_gb300 import inputs
    oracle.build()
    cores = host_cores() if oracle.has_openmp() else 1
    per_step = max(cores, 16)
    for i in range(args.warmup):
        s = inputs.query_subsample(w.m, per_step, seed=500 + i)
        oracle.aidw(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k, nthreads=cores)
    times = []
    for i in range(args.steps):
        s = inputs.query_subsample(w.m, per_step, seed=900 + i)
        t0 = time.perf_counter()
        oracle.aidw(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k, nthreads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, 1, "FP64 CPU oracle (brute-force kNN, pow)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} queries per step against all {w.n} "
                                       "data points"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- GPU timing helpers --------------------------------------------------------------

class Ctx:
    """Device-side state shared by the measurements of one run."""

    def __init__(self, dev):
        import torch

        import paper_1601_05904_gb300 as pkg
        from paper_1601_05904_gb300 import binding
        self.torch, self.pkg, self.binding, self.dev = torch, pkg, binding, dev
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        props = torch.cuda.get_device_properties(dev)
        self.sms, self.name = props.multi_processor_count, props.name
        peaks = measured_peaks() or {}
        self.peaks_source = "measured" if peaks else "fallback"
        self.sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        self.hbm = float(peaks.get("hbm_gbs", 6800.0))
        self.rates = binding.aidw_probe_pipe_rates()
        self.mix = binding.aidw_weight_mix()
        self.loop = {}
        for c in (2, 3):
            try:
                self.loop[f"{c}_ctas_per_sm"] = binding.aidw_probe_weight_loop(c)
            except binding.AidwError:
                self.loop[f"{c}_ctas_per_sm"] = None

    def tensors(self, w):
        return {k: self.torch.from_numpy(getattr(w, k)).to(self.dev)
                for k in ("x", "y", "z", "qx", "qy")}

    def time_steps(self, step, steps, warmup, clocks=None):
        """Runs warmup + steps calls of step() (L2 flushed before each timed
        one), timing each on the current stream with CUDA events and the
        library's stage events.  Returns (ms per step, stage dict, clocks)."""
        torch, binding = self.torch, self.binding
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        binding.aidw_profile_read()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        binding.aidw_profile_enable(True)
        gc.disable()   # no collection between a step's synchronous status read and its launches
        t0 = time.perf_counter()
        for i in range(steps):
            self.flush.fill_(float(i))
            ev[i][0].record()
            step()
            ev[i][1].record()
        torch.cuda.synchronize()
        self.wall = time.perf_counter() - t0
        gc.enable()
        binding.aidw_profile_enable(False)
        clk = clocks.stop() if clocks else None
        stage = binding.aidw_profile_read()
        return [a.elapsed_time(b) for a, b in ev], stage, clk

    def grid_cells(self, t, params):
        g = self.binding.aidw_grid_build(t["x"], t["y"], t["z"], params)
        info = self.binding.aidw_grid_get_info(g)
        g.destroy()
        return info["n_cells"]

    def weight_roofline(self, stage, pairs_per_launch, traffic=None):
        w_ms, w_l = stage["weight"]
        return weight_roofline(pairs_per_launch, w_ms / w_l if w_l else None, self.rates,
                               self.mix, self.sms, self.sm_mhz, traffic, self.loop)


def single_record(ctx, w, params, steps, warmup, cpu_seconds, seed, label, keep=None):
    """One workload: `steps` full steps (grid build + kNN + weighting), the
    weighting roofline, the stage rooflines and the error against the oracle
    on a query sample."""
    binding = ctx.binding
    t = ctx.tensors(w)
    out = ctx.torch.empty(w.m, dtype=ctx.torch.float32, device=ctx.dev)

    def step():
        g = binding.aidw_grid_build(t["x"], t["y"], t["z"], params)
        binding.aidw_interpolate(g, t["qx"], t["qy"], params, out_z=out)
        g.destroy()
    ms, stage, _ = ctx.time_steps(step, steps, warmup)
    ms_step = sum(ms) / len(ms)
    stage_ms = {k: v[0] / steps for k, v in stage.items()}
    rec = {"workload": label, "n_data": w.n, "n_query": w.m, "k": w.k, "steps": steps,
           "warmup": warmup, "ms_per_step": ms_step, "value": w.m / (ms_step / 1000.0),
           "unit": UNIT, "stages_ms_per_step": stage_ms,
           "roofline": ctx.weight_roofline(stage, float(w.n) * float(w.m)),
           "stage_rooflines": stage_rooflines({k: (v[0] / steps, v[1] // steps)
                                               for k, v in stage.items()},
                                              w.n, w.m, ctx.grid_cells(t, params), ctx.hbm)}
    if cpu_seconds > 0:
        s, ref, dt, cores = _oracle_sample(w, cpu_seconds, seed)
        acc = accuracy_on_sample(binding, ctx.pkg, t, w, s, ref, params, False, out.cpu().numpy())
        acc["oracle"] = f"{s.size} queries, {dt:.1f} s on {cores} cores"
        rec["accuracy"] = acc
    if keep is not None:
        keep.update(t=t, out=out)
    return rec


def precision_record(ctx, args):
    """The 4M precision form: FP32-comp on every query (timed), the plain
    FP64 GPU path on the first Q queries (the 65,536-query subsample), the
    FP32-comp against it on those Q queries, and both against the oracle on
    a sample of them."""
    from paper_1601_05904_gb300 import inputs
    torch, binding, pkg = ctx.torch, ctx.binding, ctx.pkg
    w = inputs.uniform_kilo(n=1 << 22, k=10, seed=3)
    params = pkg.Params(k=10)
    keep = {}
    rec = single_record(ctx, w, params, 2, 1, 0.0, 0, "precision form: uniform n=m=4,194,304 "
                        "in [0,1000]^2, k=10", keep)
    t, z32 = keep["t"], keep["out"]
    q = min(args.precision_fp64_queries, w.m)
    qx, qy = t["qx"][:q].contiguous(), t["qy"][:q].contiguous()
    p64 = pkg.Params(k=10, precision=binding.AIDW_FP64_PLAIN)
    g = binding.aidw_grid_build(t["x"], t["y"], t["z"], p64)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    z64, _ = binding.aidw_interpolate(g, qx, qy, p64)
    b.record()
    torch.cuda.synchronize()
    g.destroy()
    ms64 = a.elapsed_time(b)
    # S_q (the error scale) is Eq. 1 applied to |z|: the same weights, so the
    # FP32-comp path gives it to ~1e-6 relative
    zabs = t["z"].abs().contiguous()
    g = binding.aidw_grid_build(t["x"], t["y"], zabs, params)
    s_abs, _ = binding.aidw_interpolate(g, qx, qy, params)
    torch.cuda.synchronize()
    g.destroy()
    z32h, z64h, sh = z32[:q].cpu().numpy(), z64.cpu().numpy(), s_abs.cpu().numpy()
    rec["fp64_plain"] = {"queries": q, "ms": ms64, "value": q / (ms64 / 1000.0), "unit": UNIT,
                         "sample": f"first {q} of {w.m} queries against all {w.n} data points "
                                   "(kNN + weighting, grid prebuilt)"}
    rec["fp32_vs_fp64_gpu"] = dict(error_figures(z32h, z64h, sh), queries=q,
                                   measure=ERROR_MEASURE + " (S_q from the FP32-comp path on |z|)")
    s, ref, dt, cores = _oracle_sample(w, args.precision_oracle_seconds, 3030,
                                       pool=np.arange(q))
    rec["vs_oracle"] = {"queries": int(s.size), "oracle": f"{s.size} of the first {q} queries, "
                                                           f"{dt:.1f} s on {cores} cores",
                        "fp32_comp": error_figures(z32h[s], ref["z"], ref["scale"]),
                        "fp64_gpu": error_figures(z64h[s], ref["z"], ref["scale"]),
                        "tolerance": {"fp32_comp": 1e-5, "fp64": 1e-9}}
    rec["fp32_comp_over_fp64_plain"] = rec["value"] / rec["fp64_plain"]["value"]
    return rec


PAPER_SIZES = (10240, 51200, 102400, 512000, 1024000)  # 10K .. 1000K with 1K = 1024


def sweep_record(ctx):
    """The full step at the paper's sizes (uniform, data = queries)."""
    from paper_1601_05904_gb300 import inputs
    rows = []
    for n in PAPER_SIZES:
        w = inputs.uniform_kilo(n=n, k=10, seed=1)
        r = single_record(ctx, w, ctx.pkg.Params(k=10), 3 if n < 500000 else 2, 1, 0.0, 0,
                          f"uniform n=m={n}")
        rows.append({"n": n, "ms_per_step": r["ms_per_step"], "value": r["value"],
                     "stages_ms_per_step": r["stages_ms_per_step"],
                     "weight_frac": r["roofline"]["frac"]})
    return {"workload": "uniform n=m in [0,1000]^2, k=10, the paper's sizes (1K = 1024)",
            "unit": UNIT, "rows": rows}


def batch_measure(ctx, n_jobs, steps, warmup, tune, seed_base=1000, clocks=None,
                  oracle_jobs=0, oracle_queries=32):
    """Batched form: n_jobs independent jobs of uneven size per step (grid
    builds, kNN and weighting of all jobs as one CUDA-graph replay)."""
    from paper_1601_05904_gb300 import inputs
    torch, binding, pkg = ctx.torch, ctx.binding, ctx.pkg
    ws = inputs.batch_jobs(n_jobs=n_jobs, seed_base=seed_base)
    jobs = [binding.BatchJob(*(torch.from_numpy(getattr(w, a)).to(ctx.dev)
                               for a in ("x", "y", "z", "qx", "qy")), w.k) for w in ws]
    params = pkg.Params(k=10)
    plan = binding.aidw_batch_plan_create(jobs, params)
    t0 = time.perf_counter()
    tune_ms = binding.aidw_batch_plan_tune(plan, jobs) if tune else None
    tune_s = time.perf_counter() - t0
    info = binding.aidw_batch_plan_get(plan)
    info["classes"] = binding.aidw_batch_plan_get_classes(plan)
    ms, _, clk = ctx.time_steps(lambda: binding.aidw_batch_run(plan, jobs), steps, warmup,
                                clocks)
    if binding.aidw_batch_plan_status(plan) != 0:
        raise RuntimeError("batch run reported a device error")
    step_ms = sum(ms) / len(ms)
    total_q = sum(w.m for w in ws)
    pairs = float(info["total_pairs"])
    b = weight_pair_bounds(ctx.rates, ctx.mix)
    peak = b["own_mix"] * ctx.sms * ctx.sm_mhz * 1e6
    rec = {"workload": f"batch of {n_jobs} jobs, n_j = m_j log-uniform in [1e3, 2e5], "
                       "k_j in {8,10,16,24,32}, per-job uniform + Gaussian-cluster mix in "
                       "[0,1000]^2",
           "steps": steps, "warmup": warmup, "ms_per_step": step_ms,
           "value": total_q / (step_ms / 1000.0), "unit": UNIT,
           "total_data_points": int(sum(w.n for w in ws)), "total_queries": total_q,
           "total_pairs": int(pairs), "pairs_per_s": pairs / (step_ms / 1000.0),
           "plan": dict(info, tune_build_knn_ms=tune_ms, tune_seconds=tune_s),
           "roofline": {"bound": "alu", "kernel": "whole batch step (graph: builds, kNN, "
                                                  "one persistent weighting launch)",
                        "achieved": pairs / (step_ms / 1000.0) / 1e9, "peak": peak / 1e9,
                        "unit": "Gpair/s", "frac": pairs / (step_ms / 1000.0) / peak,
                        "traffic": None, "peak_basis": "own-mix ceiling of k_weight_f32"}}
    if oracle_jobs > 0:
        import oracle
        oracle.build()
        cores = host_cores() if oracle.has_openmp() else 1
        sel = np.linspace(0, n_jobs - 1, min(oracle_jobs, n_jobs)).round().astype(int)
        worst = {"max_norm_err": 0.0, "max_rel_err_large": 0.0}
        nq = 0
        for j in sel:
            w = ws[j]
            s = inputs.query_subsample(w.m, oracle_queries, seed=7000 + int(j))
            ref = oracle.aidw(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k, nthreads=cores)
            f = error_figures(jobs[j].out_z.cpu().numpy()[s], ref["z"], ref["scale"])
            worst["max_norm_err"] = max(worst["max_norm_err"], f["max_norm_err"])
            worst["max_rel_err_large"] = max(worst["max_rel_err_large"], f["max_rel_err_large"])
            nq += s.size
        rec["accuracy"] = dict(worst, queries=nq, jobs=[int(j) for j in sel],
                               tolerance={"fp32_comp": 1e-5}, measure=ERROR_MEASURE)
    plan.destroy()
    return rec, clk


def run_configs(ctx, args, headline_pairs_per_s):
    """Every other workload, each with its own steps, roofline and oracle
    error; a failure of one is recorded and does not stop the others."""
    from paper_1601_05904_gb300 import inputs
    out = {}

    def guard(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # recorded, not hidden
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
        ctx.torch.cuda.synchronize()

    for k in (10, 20):
        guard(f"clustered_k{k}", lambda k=k: single_record(
            ctx, inputs.clustered_kilo(n=1 << 20, k=k, seed=2), ctx.pkg.Params(k=k), 3, 1,
            args.sub_cpu_seconds, 5050 + k,
            f"clustered n=m=1,048,576 (32 Gaussians + 10 % uniform), k={k}"))
    guard("precision_4M", lambda: precision_record(ctx, args))

    def batch():
        rec, _ = batch_measure(ctx, args.jobs, 3, 1, True, oracle_jobs=16)
        rec["pair_rate_vs_single_job"] = rec["pairs_per_s"] / headline_pairs_per_s
        return rec
    guard("batch_512", batch)
    guard("sweep", lambda: sweep_record(ctx))
    return out


# ---- the headline line -------------------------------------------------------------

def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1601_05904_gb300 import binding
    binding.load()
    ctx = Ctx(dev)
    pkg = ctx.pkg
    strong = args.scaling == "strong" and world > 1

    w = make_workload(args, rank, args.scaling)
    params = pkg.Params(k=w.k, cell_scale=args.cell_scale)
    t = ctx.tensors(w)
    out_z = torch.full((w.m,), float("nan"), dtype=torch.float32, device=dev)
    robs = torch.empty(w.m, dtype=torch.float32, device=dev)
    q_lo, q_hi = binding.aidw_shard_range(w.m, rank, world) if strong else (0, w.m)
    my_q = q_hi - q_lo

    def step():
        g = binding.aidw_grid_build(t["x"], t["y"], t["z"], params)
        if args.mode == "knn":
            binding.aidw_knn(g, t["qx"], t["qy"], w.k, out_robs=robs, want=("robs",))
        elif args.mode == "local":
            binding.aidw_interpolate_local(g, t["qx"], t["qy"], params, out_z=out_z)
        elif strong:
            binding.aidw_interpolate_shard(g, t["qx"], t["qy"], rank, world, params, out_z=out_z)
        else:
            binding.aidw_interpolate(g, t["qx"], t["qy"], params, out_z=out_z)
        g.destroy()

    if world > 1:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    ms, stage, clk = ctx.time_steps(step, args.steps, args.warmup if world == 1 else 0, clocks)
    wall = ctx.wall
    if world > 1:
        torch.distributed.barrier()
    step_ms = sum(ms) / args.steps
    my_s = max_over_ranks(step_ms * args.steps / 1000.0, dev)
    value = (strong_value(w.m, args.steps, my_s) if strong
             else whole_job_value(world, w.m, args.steps, my_s))
    launches = sum(v[1] for v in stage.values())

    # float64 plain path on a query sample (kNN + weighting, grid prebuilt)
    fp64 = None
    if args.fp64_queries > 0 and rank == 0 and args.mode != "knn":
        interp = (binding.aidw_interpolate_local if args.mode == "local"
                  else binding.aidw_interpolate)
        mq = min(args.fp64_queries, w.m)
        p64 = pkg.Params(k=w.k, precision=binding.AIDW_FP64_PLAIN)
        qx64, qy64 = t["qx"][:mq].contiguous(), t["qy"][:mq].contiguous()
        g = binding.aidw_grid_build(t["x"], t["y"], t["z"], p64)
        interp(g, qx64, qy64, p64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        interp(g, qx64, qy64, p64)
        b.record()
        torch.cuda.synchronize()
        g.destroy()
        ms64 = a.elapsed_time(b)
        fp64 = {"value": mq / (ms64 / 1000.0), "unit": UNIT,
                "sample": f"first {mq} of {w.m} queries against all {w.n} data points "
                          "(kNN + weighting, grid prebuilt)",
                "ms": ms64}

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0 and args.mode == "aidw":
        host = {k: torch.from_numpy(getattr(w, k)).pin_memory() for k in ("x", "y", "z")}
        host["qx"] = torch.from_numpy(w.qx[q_lo:q_hi].copy()).pin_memory()
        host["qy"] = torch.from_numpy(w.qy[q_lo:q_hi].copy()).pin_memory()
        binding.interpolate_host(host["x"], host["y"], host["z"], host["qx"], host["qy"], params)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            zh = binding.interpolate_host(host["x"], host["y"], host["z"], host["qx"],
                                          host["qy"], params)
            float(zh[0])
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
        h2d = sum(v.numel() * 4 for v in host.values())
        e2e = {"value": (strong_value(w.m, args.e2e_steps, e2e_s) if strong
                         else whole_job_value(world, w.m, args.e2e_steps, e2e_s)),
               "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(my_q * 4),
               "ms_per_step": 1000.0 * e2e_s / args.e2e_steps}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    pairs = float(w.n) * float(my_q)
    traffic = WEIGHT_DRAM_BYTES_PER_POINT * w.n if (w.n == w.m and not strong) else None
    roofline = ctx.weight_roofline(stage, pairs, traffic)
    roofline["traffic_basis"] = "dram bytes per launch, ncu at n = m = 131072 scaled by n"
    if args.mode in ("local", "knn"):
        # kNN + local weighting in one kernel: algorithmic bytes are the
        # queries (8 B in, 4 B out) and the data set read once (16 B points
        # + 4 B z + 4 B cell head per point)
        k_ms, k_launches = stage["knn"]
        alg = 12.0 * w.m + 24.0 * w.n
        ach = alg / (k_ms / k_launches / 1000.0) / 1e9 if k_launches else None
        roofline = {"bound": "hbm", "kernel": "k_knn (grid kNN" +
                    (" + local weighting)" if args.mode == "local" else ")"),
                    "achieved": ach, "peak": ctx.hbm, "unit": "GB/s",
                    "frac": (ach / ctx.hbm) if ach else None, "traffic": None,
                    "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy); the kernel is bound by "
                                  "dependent L2 gathers of the ring search, not by HBM"}
    stages_ms = {k: v[0] / args.steps for k, v in stage.items()}
    st_roof = stage_rooflines({k: (v[0] / args.steps, v[1] // args.steps)
                               for k, v in stage.items()}, w.n, my_q,
                              ctx.grid_cells(t, params), ctx.hbm)
    cpu = None
    accuracy = None
    if not args.no_cpu_baseline and world == 1:     # the oracle on rank 0 at N = 1 only
        cpu, sample, ref = cpu_baseline(w, args.cpu_seconds, rank, local=args.mode == "local")
        if args.mode in ("aidw", "local"):
            accuracy = accuracy_on_sample(binding, pkg, t, w, sample, ref, params,
                                          args.mode == "local", out_z.cpu().numpy())
    configs = None
    if (args.configs == "all" and world == 1 and args.mode == "aidw"
            and args.workload == "uniform" and args.n == 1 << 20):
        configs = run_configs(ctx, args, pairs / (step_ms / 1000.0))
    metric = {"aidw": METRIC,
              "local": "local AIDW interpolated points/s at n=m=1M (kNN + Eq. 1 over the k nearest)",
              "knn": "grid build + kNN queries/s at n=m=1M (r_obs per query)"}[args.mode]
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, world, scaling=args.scaling),
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "stage_rooflines": st_roof, "cpu_baseline": cpu, "accuracy": accuracy,
            "fp64_plain": fp64, "stages_ms_per_step": stages_ms, "wall_s_timed": wall,
            "clocks": clk, "device": ctx.name, "peaks": ctx.peaks_source}
    if fp64 and args.mode == "aidw":
        line["fp32_comp_over_fp64_plain"] = value / fp64["value"]
    if configs is not None:
        line["configs"] = configs
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """The batched form as the line's own workload."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1601_05904_gb300 import binding
    binding.load()
    ctx = Ctx(dev)
    if world > 1:
        torch.distributed.barrier()
    rec, clk = batch_measure(ctx, args.jobs, args.steps, args.warmup, not args.no_tune,
                             seed_base=1000 + 100_000 * rank, clocks=ClockSampler(local))
    step_s = max_over_ranks(rec["ms_per_step"] / 1000.0, dev)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    line = {"metric": "AIDW batched interpolated points/s (512 jobs, n_j log-uniform 1e3..2e5)",
            "value": whole_job_value(world, rec["total_queries"], 1, step_s), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": rec["workload"], "total_data_points": rec["total_data_points"],
                       "total_queries": rec["total_queries"], "total_pairs": rec["total_pairs"],
                       "plan": rec["plan"],
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
            "pairs_per_s": rec["pairs_per_s"], "roofline": rec["roofline"],
            "clocks": clk, "device": ctx.name}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# DRAM bytes (read + write) of one k_weight_f32 launch per data point, from
# the ncu capture at n = m = 131,072 (5.82 MB read, 0 written); every input
# (points, queries, kNN records) is read once, so it scales with n = m.
WEIGHT_DRAM_BYTES_PER_POINT = 5.821696e6 / 131072


def _time_ms(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_tables(args):
    """Per-size tables at the paper's sizes (uniform data = queries in a square)."""
    import torch

    import paper_1601_05904_gb300 as pkg
    from paper_1601_05904_gb300 import binding, inputs

    torch.cuda.set_device(0)
    binding.load()
    dev = torch.device("cuda", 0)
    rows = []
    for n in PAPER_SIZES:
        w = inputs.uniform_kilo(n=n, k=args.k, seed=1)
        t = {a: torch.from_numpy(getattr(w, a)).to(dev) for a in ("x", "y", "z", "qx", "qy")}
        p = pkg.Params(k=w.k)
        if args.mode == "knn-table":
            def grid_knn():
                g = binding.aidw_grid_build(t["x"], t["y"], t["z"], p)
                binding.aidw_knn(g, t["qx"], t["qy"], w.k, want=("robs",))
                g.destroy()
            g = binding.aidw_grid_build(t["x"], t["y"], t["z"], p)

            def brute():
                binding.aidw_knn_bruteforce(g, t["qx"], t["qy"], w.k, want=("robs",))
            reps = max(1, args.steps)
            ms_grid = _time_ms(grid_knn, reps)
            ms_brute = _time_ms(brute, 1 if n > 200000 else reps)
            g.destroy()
            rows.append({"n": n, "grid_build_plus_knn_ms": ms_grid, "all_points_knn_ms": ms_brute,
                         "speedup": ms_brute / ms_grid})
        else:
            def step():
                g = binding.aidw_grid_build(t["x"], t["y"], t["z"], p)
                binding.aidw_interpolate(g, t["qx"], t["qy"], p)
                g.destroy()
            ms = _time_ms(step, max(1, args.steps if n < 500000 else 2))
            rows.append({"n": n, "ms": ms, "points_per_s": n / (ms / 1000.0)})
    metric = ("kNN stage time, grid search vs all-points search (paper Table 3 sizes)"
              if args.mode == "knn-table" else
              "AIDW step time at the paper's sizes (paper Table 1 sizes)")
    print(json.dumps({"metric": metric, "unit": "ms", "k": args.k, "data": "synthetic uniform",
                      "device": torch.cuda.get_device_properties(dev).name, "rows": rows}),
          flush=True)
    return 0


def run_knn_rule(args):
    """How often the paper's level rule (Sec. 3.2.4: first level holding k
    points, plus one) misses a true neighbour, against the exact grid kNN on
    the same grid: share of queries whose k-nearest list differs, r_obs
    (Eq. 3) error, and the time of both searches."""
    import torch

    import paper_1601_05904_gb300 as pkg
    from paper_1601_05904_gb300 import binding, inputs

    torch.cuda.set_device(0)
    binding.load()
    dev = torch.device("cuda", 0)
    rows = []
    for wname in ("uniform", "clustered"):
        gen = inputs.uniform_kilo if wname == "uniform" else inputs.clustered_kilo
        w = gen(n=args.n, k=args.k)
        t = {a: torch.from_numpy(getattr(w, a)).to(dev) for a in ("x", "y", "z", "qx", "qy")}
        for cs in (1.0, 0.0):
            p = pkg.Params(k=w.k, cell_scale=cs)
            g = binding.aidw_grid_build(t["x"], t["y"], t["z"], p)
            ie, _, re_ = binding.aidw_knn(g, t["qx"], t["qy"], w.k)
            ip, _, rp = binding.aidw_knn_paper_rule(g, t["qx"], t["qy"], w.k)
            torch.cuda.synchronize()
            differ = (ie != ip).any(dim=1)
            rel = ((rp.double() - re_.double()) / re_.double().clamp_min(1e-300)).abs()
            reps = max(1, args.steps)
            ms_exact = _time_ms(lambda: binding.aidw_knn(g, t["qx"], t["qy"], w.k,
                                                         want=("robs",)), reps)
            ms_paper = _time_ms(lambda: binding.aidw_knn_paper_rule(g, t["qx"], t["qy"], w.k,
                                                                    want=("robs",)), reps)
            info = binding.aidw_grid_get_info(g)
            assert binding.aidw_grid_status(g) == 0
            g.destroy()
            rows.append({"workload": wname, "cell_scale": info["cell_scale"],
                         "cell_width": info["cell_width"],
                         "queries_with_a_missed_neighbour": float(differ.double().mean()),
                         "r_obs_rel_err_max": float(rel.max()),
                         "r_obs_rel_err_mean": float(rel.mean()),
                         "exact_knn_ms": ms_exact, "paper_rule_knn_ms": ms_paper})
    print(json.dumps({"metric": "kNN misses of the paper's level rule vs the exact grid kNN",
                      "n": args.n, "k": args.k, "data": "synthetic",
                      "device": torch.cuda.get_device_properties(dev).name, "rows": rows}),
          flush=True)
    return 0


def main(argv=None):
    args = parse(argv)
    # oracle time of each sub-record's accuracy check and of the 4M form
    args.sub_cpu_seconds = min(4.0, args.cpu_seconds)
    args.precision_oracle_seconds = min(8.0, 2 * args.cpu_seconds)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.mode in ("knn-table", "sweep"):
        return run_tables(args)
    if args.mode == "knn-rule":
        return run_knn_rule(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
