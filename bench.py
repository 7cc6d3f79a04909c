"""Throughput of the AIDW hot path (grid build + grid kNN + all-points
weighting) on GB300, printed as one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole path over one batch: build the even grid of
the data points, find every query's k nearest neighbours, compute alpha and
the weighted prediction of Eq. 1 over all data points.  The default workload
is n = m = 1,048,576 points uniform in [0,1000]^2, k = 10, float32 with
compensated sums (AIDW_FP32_COMP).

Under torchrun (N > 1) every rank runs the same-sized workload on its own
GPU with its own seeded queries against the same data (weak scaling: the
queries shard, nothing is exchanged on the data path); rank 0 prints the
total over ranks divided by the slowest rank's time.

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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=1 << 20, help="data points = queries")
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--workload", choices=("uniform", "clustered", "batch"), default="uniform")
    ap.add_argument("--jobs", type=int, default=512, help="jobs of the batch workload")
    ap.add_argument("--no-tune", action="store_true", help="batch: skip the autotuner")
    ap.add_argument("--cell-scale", type=float, default=0.0,
                    help="grid cell width / r_exp (<= 0: the library's choice)")
    ap.add_argument("--mode", choices=("aidw", "local", "knn", "knn-table", "sweep", "knn-rule"),
                    default="aidw",
                    help="aidw: Eq. 1 over all points; local: Eq. 1 over the k nearest; "
                         "knn-table: grid vs all-points kNN at the paper's sizes; "
                         "sweep: the full step at the paper's sizes")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-queries", type=int, default=16384)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


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


def make_workload(args, rank):
    from paper_1601_05904_gb300 import inputs
    if args.workload == "uniform":
        w = inputs.uniform_kilo(n=args.n, k=args.k, seed=1)
    else:
        w = inputs.clustered_kilo(n=args.n, k=args.k, seed=2)
    if rank:
        # each rank its own queries over the same data (weak scaling)
        rng = np.random.default_rng(10_000 + rank)
        w.qx, w.qy = inputs.uniform_points(rng, w.m, 0.0, inputs.SIDE_KILO)
    return w


def workload_config(args, world, precision=None):
    return {"workload": f"{args.workload} n=m={args.n} in [0,1000]^2, k={args.k}, "
                        "alpha levels 1..5, R_min/R_max 0/2",
            "n_data": args.n, "n_query_per_gpu": args.n, "k": args.k,
            "precision": precision or "FP32-comp (SFU exp2/log2, TwoSum-compensated f32 "
                                      "sums, f64 final divide; alpha in f32 with a "
                                      "compensated r_obs sum)",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "parallelism": f"query-sharded x{world}" if world > 1 else "single GPU"}


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


def cpu_baseline(w, seconds: float, rank: int, local: bool = False):
    """The oracle as it stands, on the host cores, over a bounded query sample.
    Returns (baseline dict, sample indices, oracle results on the sample)."""
    import oracle
    from paper_1601_05904_gb300 import inputs
    oracle.build()
    fn = oracle.aidw_local if local else oracle.aidw
    cores = host_cores() if oracle.has_openmp() else 1
    probe = max(cores, 8)
    s = inputs.query_subsample(w.m, probe, seed=2024 + rank)
    t0 = time.perf_counter()
    fn(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k, nthreads=cores)
    per_q = (time.perf_counter() - t0) / probe
    count = int(max(probe, min(w.m, seconds / max(per_q, 1e-9))))
    s = inputs.query_subsample(w.m, count, seed=4048 + rank)
    t0 = time.perf_counter()
    ref = fn(w.x, w.y, w.z, w.qx[s], w.qy[s], w.k, nthreads=cores)
    dt = time.perf_counter() - t0
    return ({"value": count / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"{count} of {w.m} queries against all {w.n} data points "
                       f"({dt:.1f} s, FP64, brute-force kNN with full sort)"}, s, ref)


def accuracy_on_sample(binding, pkg, t, w, s, ref, params, local, z32_all):
    """Error of the GPU predictions against the oracle on the baseline's
    sample: max |z - z_ref| / S_q (S_q = sum w|z| / sum w) for the FP32-comp
    output of the timed steps and for the FP64 path run on the same queries,
    and the largest alpha difference."""
    import oracle
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
    e32 = oracle.normalized_error(z32_all[s], ref["z"], ref["scale"])
    e64 = oracle.normalized_error(z64.cpu().numpy(), ref["z"], ref["scale"])
    ea = np.abs(a32.cpu().numpy().astype(np.float64) - ref["alpha"])
    return {"queries": int(s.size), "fp32_comp_max_norm_err": float(e32.max()),
            "fp32_comp_mean_norm_err": float(e32.mean()), "fp64_max_norm_err": float(e64.max()),
            "alpha_max_abs_err": float(ea.max()),
            "tolerance": {"fp32_comp": 1e-5, "fp64": 1e-9},
            "measure": "max_q |z - z_oracle| / S_q, S_q = sum w|z| / sum w (oracle)"}


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
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, 1, "FP64 CPU oracle (brute-force kNN, pow)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} queries per step against all {w.n} "
                                       "data points"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    import paper_1601_05904_gb300 as pkg
    from paper_1601_05904_gb300 import binding

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    binding.load()

    w = make_workload(args, rank)
    params = pkg.Params(k=w.k, cell_scale=args.cell_scale)
    t = {k: torch.from_numpy(getattr(w, k)).to(dev) for k in ("x", "y", "z", "qx", "qy")}
    out_z = torch.empty(w.m, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    interp = (binding.aidw_interpolate_local if args.mode == "local"
              else binding.aidw_interpolate)
    robs = torch.empty(w.m, dtype=torch.float32, device=dev)

    def step():
        g = binding.aidw_grid_build(t["x"], t["y"], t["z"], params)
        if args.mode == "knn":
            binding.aidw_knn(g, t["qx"], t["qy"], w.k, out_robs=robs, want=("robs",))
        else:
            interp(g, t["qx"], t["qy"], params, out_z=out_z)
        g.destroy()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    binding.aidw_profile_read()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    binding.aidw_profile_enable(True)
    gc.disable()   # no collection between a step's synchronous status read and its launches
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        step()
        ev[i][1].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    gc.enable()
    binding.aidw_profile_enable(False)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    stage = binding.aidw_profile_read()
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    my_s = max_over_ranks(step_ms * args.steps / 1000.0, dev)
    value = whole_job_value(world, w.m, args.steps, my_s)
    launches = sum(v[1] for v in stage.values())

    # float64 plain path on a query sample (kNN + weighting + grid build)
    fp64 = None
    if args.fp64_queries > 0 and rank == 0 and args.mode != "knn":
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
        ms = a.elapsed_time(b)
        fp64 = {"value": mq / (ms / 1000.0), "unit": UNIT,
                "sample": f"first {mq} of {w.m} queries against all {w.n} data points "
                          "(kNN + weighting, grid prebuilt)",
                "ms": ms}

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        host = {k: torch.from_numpy(getattr(w, k)).pin_memory() for k in ("x", "y", "z", "qx", "qy")}
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
        e2e = {"value": whole_job_value(world, w.m, args.e2e_steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(w.m * 4),
               "ms_per_step": 1000.0 * e2e_s / args.e2e_steps}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks() or {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    w_ms, w_launches = stage["weight"]
    pairs = float(w.n) * float(w.m)
    achieved = pairs / (w_ms / w_launches / 1000.0) / 1e9 if w_launches else None
    # Every (query, data point) pair needs one SFU log2 and one SFU exp2; the
    # two share the SFU pipe, so the pipe bounds the pair rate at
    # 1 / (1/r_lg2 + 1/r_ex2) per SM per clock (rates measured live).
    rates = binding.aidw_probe_pipe_rates()
    pairs_per_sm_clk = 1.0 / (1.0 / rates["lg2"] + 1.0 / rates["ex2"])
    peak = pairs_per_sm_clk * props.multi_processor_count * sm_max * 1e6 / 1e9
    traffic = WEIGHT_DRAM_BYTES_PER_POINT * w.n if w.n == w.m else None
    roofline = {"bound": "alu", "kernel": "k_weight_f32 (all-points weighting, Eq. 1)",
                "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_basis": "dram bytes per launch, ncu at n = m = 131072 scaled by n",
                "peak_basis": (f"SFU pipe: measured lg2 {rates['lg2']:.2f} and ex2 "
                               f"{rates['ex2']:.2f} per SM per clock -> "
                               f"{pairs_per_sm_clk:.2f} pairs per SM per clock x "
                               f"{props.multi_processor_count} SMs x {sm_max:.0f} MHz max clock"),
                "pipe_rates_per_sm_clk": rates}
    if args.mode in ("local", "knn"):
        # kNN + local weighting in one kernel: algorithmic bytes are the
        # queries (8 B in, 4 B out) and the data set read once (16 B points
        # + 4 B z + 4 B cell head per point)
        k_ms, k_launches = stage["knn"]
        alg = 12.0 * w.m + 24.0 * w.n
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        ach = alg / (k_ms / k_launches / 1000.0) / 1e9 if k_launches else None
        roofline = {"bound": "hbm", "kernel": "k_knn (grid kNN" +
                    (" + local weighting)" if args.mode == "local" else ")"),
                    "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": (ach / hbm) if ach else None, "traffic": None,
                    "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy); the kernel is bound by "
                                  "dependent L2 gathers of the ring search, not by HBM"}
    stages_ms = {k: v[0] / args.steps for k, v in stage.items()}
    cpu = None
    accuracy = None
    if not args.no_cpu_baseline and world == 1:     # the oracle on rank 0 at N = 1 only
        cpu, sample, ref = cpu_baseline(w, args.cpu_seconds, rank, local=args.mode == "local")
        if args.mode in ("aidw", "local"):
            accuracy = accuracy_on_sample(binding, pkg, t, w, sample, ref, params,
                                          args.mode == "local", out_z.cpu().numpy())
    metric = {"aidw": METRIC,
              "local": "local AIDW interpolated points/s at n=m=1M (kNN + Eq. 1 over the k nearest)",
              "knn": "grid build + kNN queries/s at n=m=1M (r_obs per query)"}[args.mode]
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args, world),
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "cpu_baseline": cpu, "accuracy": accuracy, "fp64_plain": fp64,
            "stages_ms_per_step": stages_ms, "wall_s_timed": wall,
            "clocks": clk, "device": props.name}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """Batched form: many independent jobs of uneven size per step (grid
    builds, kNN and weighting of all jobs as one CUDA-graph replay)."""
    import torch

    import paper_1601_05904_gb300 as pkg
    from paper_1601_05904_gb300 import binding, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    binding.load()
    ws = inputs.batch_jobs(n_jobs=args.jobs, seed_base=1000 + 100_000 * rank)
    jobs = [binding.BatchJob(*(torch.from_numpy(getattr(w, a)).to(dev)
                               for a in ("x", "y", "z", "qx", "qy")), w.k) for w in ws]
    params = pkg.Params(k=10)
    plan = binding.aidw_batch_plan_create(jobs, params)
    tune_ms = None if args.no_tune else binding.aidw_batch_plan_tune(plan, jobs)
    info = binding.aidw_batch_plan_get(plan)
    for _ in range(args.warmup):
        binding.aidw_batch_run(plan, jobs)
    torch.cuda.synchronize()
    if binding.aidw_batch_plan_status(plan) != 0:
        raise RuntimeError("batch run reported a device error")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    gc.disable()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        binding.aidw_batch_run(plan, jobs)
        ev[i][1].record()
    torch.cuda.synchronize()
    gc.enable()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = 1000.0 * max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1000.0,
                                      dev) / args.steps
    total_q = sum(w.m for w in ws)
    if rank != 0:
        plan.destroy()
        torch.distributed.destroy_process_group()
        return 0
    rates = binding.aidw_probe_pipe_rates()
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks() or {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = 1.0 / (1.0 / rates["lg2"] + 1.0 / rates["ex2"]) * props.multi_processor_count * sm_max * 1e6
    pairs = float(info["total_pairs"])
    line = {"metric": "AIDW batched interpolated points/s (512 jobs, n_j log-uniform 1e3..2e5)",
            "value": whole_job_value(world, total_q, 1, step_ms / 1000.0), "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"batch of {args.jobs} jobs, n_j = m_j log-uniform in "
                                   "[1e3, 2e5], k_j in {8,10,16,24,32}, per-job uniform + "
                                   "Gaussian-cluster mix in [0,1000]^2",
                       "total_data_points": int(sum(w.n for w in ws)), "total_queries": total_q,
                       "total_pairs": int(pairs), "cell_scale": info["cell_scale"],
                       "knn_threads": info["knn_threads"], "tune_build_knn_ms": tune_ms,
                       "pool_bytes": info["pool_bytes"],
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
            "pairs_per_s": pairs / (step_ms / 1000.0),
            "roofline": {"bound": "alu", "kernel": "whole batch step (graph)",
                         "achieved": pairs / (step_ms / 1000.0) / 1e9, "peak": peak / 1e9,
                         "unit": "Gpair/s", "frac": pairs / (step_ms / 1000.0) / peak,
                         "traffic": None},
            "clocks": clk, "device": props.name}
    plan.destroy()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


PAPER_SIZES = (10240, 51200, 102400, 512000, 1024000)  # 10K .. 1000K with 1K = 1024

# DRAM bytes (read + write) of one k_weight_f32 launch per data point, from
# the ncu capture at n = m = 131,072 (5.80 MB read, 0 written); every input
# (points, queries, kNN records) is read once, so it scales with n = m.
WEIGHT_DRAM_BYTES_PER_POINT = 5.82144e6 / 131072


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


def main():
    args = parse()
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
