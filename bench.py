"""Benchmark of the collision-integral hot path on GB300.

Workload (default): the 2->2 Bose-Einstein problem with massless and
m = 0.5 scalars, 128 log-spaced grid points on [1e-3, 30], sigma_E = 0.005,
1e6 samples per task per iteration x 8 iterations (512 tasks: 2 species x
128 points x gain/loss), f = BE(T=1) + a Gaussian bump, stepped with Heun.
One bench step = one Heun step = two full collision sweeps (spline build,
8 VEGAS iterations of the persistent sample kernel + refinement, assembly)
plus the predictor and corrector updates.

Metric: C[f] grid sweeps/s (FP32 integrand path) at the configured budget;
also integrand evals/s, the FP64 path, and both normalised to a 1e-4 median
relative MC error of the gain / loss estimates.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "C[f] grid sweeps/s and integrand evals/s, FP32 vs FP64 path, at 1e-4 rel MC err"
UNIT = "sweeps/s"
WORKLOAD = "c2_bose_2to2"
DT = 0.5          # requested Heun step (bounded by Eq. (16) inside each step)
CPU_NEVAL = 20_000  # samples per iteration of the oracle tasks timed on the host
# DRAM bytes per sample-kernel launch (dram__bytes_read.sum + dram__bytes_write.sum) and thread
# instructions per sample (smsp__inst_executed.sum x 32 / samples: issue slots in thread units) of the
# 2->2 Bose sample kernel, from one ncu capture of a timed-step launch of this kernel version at
# 5e5 samples per task (summarised under profiles/); the tables it reads do not grow with
# the sample count.  The kernel is issue-bound, so its instruction issue rate against the SMs' issue peak
# says how close it is to the hardware limit.
TRAFFIC_BYTES_PER_LAUNCH = 1.903872e6
INSTR_PER_SAMPLE_C2 = 310.4
# FP32 FLOP per sample measured by ncu's FP32 operation counters (FFMA, FADD, FMUL and their packed
# FP32x2 forms) on the same launch shape: the source count charges every sample the statistical
# factor, which the per-warp queue evaluates only for near-shell samples.
MEASURED_FLOPS_PER_SAMPLE_C2 = 122.9
ISSUE_PEAK_TINSTR = 152 * 4 * 32 * 2.07e9 / 1e12     # 4 schedulers x 1 warp instruction / clock
FP32_PEAK_TFLOPS_NOMINAL = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def flops_per_sample(n_legs):
    """FP32 operations per sample of the sample kernel, counted from its
    source (FMA = 2): 5 per VEGAS dimension (3 per integrated leg), 33 per
    integrated leg (sincos argument scaling, momentum components, energy,
    energy balance, measure, spline lookup, statistical factor), 23 for the
    conserved leg, 2 for the Gaussian argument, 4 + 1 for the weight and its
    square and 8 for the two compensated sums:  48 (n - 2) + 40."""
    return 48 * (n_legs - 2) + 40


def mufu_per_sample(n_legs):
    """Special-function-unit operations per sample: 2 sincos + 1 rsqrt +
    1 log2 per integrated leg, 2 rsqrt + 1 log2 for the conserved leg and the
    Gaussian's exp2."""
    return 6 * (n_legs - 2) + 4


NEVAL = None      # per-task samples per iteration; None = the workload's own
WORKLOAD_KEY = "c2"
STRAT = False     # stratified sampling (VEGAS+) in every process
VARB = False      # variance-driven per-task budgets (multi-species workload)
# per workload: (builder, integrator, requested dt, start time, description)
WORKLOADS = {
    "c1": ("c1_maxwell_2to2", "euler", 0.1, 0.0,
           "MB 2->2, m=1, 32 log points [0.01,20], sigma_E=0.01, 1e4 samples x 5 iterations, Euler dt=0.1"),
    "c2": ("c2_bose_2to2", "heun", 0.5, 0.0,
           "2 species (m=0, m=0.5) BE 2->2, 128 log points [1e-3,30], sigma_E=0.005, 1e6 samples x 8 "
           "iterations per task, 512 tasks, Heun steps"),
    "c3": ("c3_cannibal_2to3", "heun", 0.5, 0.0,
           "BE 2<->3 m=1 (both pinned sides) + 2->2, 256 log points [0.01,25], sigma_E=0.01, 4e6 x 10, Heun"),
    "c4": ("c4_multi_species", "heun", 0.5, 1.0,
           "A (BE, m=1+0.1t) + B (FD, m=0.3): AB->AB, AA->AAA, AAA->BB, FRW a=(t/t0)^1/2, 512 log points "
           "[0.01,25], budgets 1e5..1e7 per point x 2 iterations, Heun from t=1"),
    "c5": ("c5_2to4", "heun", 0.5, 0.0,
           "BE 2->4 m=1 (12-dim), 256 log points [0.01,25], sigma_E=0.01, 2e6 x 2, Heun + adjoint"),
}


def workload():
    prob, f0 = _workload()
    if STRAT:
        from dataclasses import replace
        prob = replace(prob, processes=tuple(replace(p, strat=1) for p in prob.processes))
    return prob, f0


def _workload():
    import workloads as W
    name = WORKLOADS[WORKLOAD_KEY][0]
    fn = getattr(W, name)
    if WORKLOAD_KEY == "c4":
        kw = dict(variance_budgets=VARB)
        if NEVAL is not None:
            kw.update(nmin=NEVAL, nmax=NEVAL * 100)
        return fn(**kw)
    if NEVAL is not None:
        if WORKLOAD_KEY == "c3":
            return fn(neval=NEVAL, with_2to2=True)
        return fn(neval=NEVAL)
    if WORKLOAD_KEY == "c3":
        return fn(with_2to2=True)
    return fn()


def mean_flops_per_sample(prob, col):
    """Sample-weighted FP32 FLOP count over the processes of a problem."""
    n = prob.grid.n
    tot = 0.0
    cnt = 0.0
    for p in prob.processes:
        legs = len(p.species_in) + len(p.species_out)
        sym = sorted(p.species_in) == sorted(p.species_out)
        sides = len(set(p.species_in)) + (0 if sym else len(set(p.species_out)))
        per = p.neval_per_point if p.neval_per_point is not None else [p.neval] * n
        s = 2 * sides * sum(per)
        tot += s * flops_per_sample(legs)
        cnt += s
    return tot / cnt, max(len(p.species_in) + len(p.species_out) for p in prob.processes)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def rel_err_stats(col):
    mean, err = col.task_results()
    ok = np.abs(mean) > 0
    r = err[ok] / np.abs(mean[ok])
    return float(np.median(r)), float(np.max(r))


def run_native(args, rank, world):
    import torch

    import workloads as W
    from paper_2603_28848_gb300 import Collision, build

    build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    prob, f0 = workload()
    wl = WORKLOADS[WORKLOAD_KEY]
    method, DT, T0 = wl[1], wl[2], wl[3]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MiB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---------------- FP32 path: the headline ----------------------------------------
    # Heun steps replayed from a CUDA graph (best_evolve) after the launch
    # shape was picked by the autotuner (best_autotune).
    col = Collision(prob, W.PREC_FP32)
    col_tasks = col.n_tasks
    evals = col.sweep_samples()
    samples_per_launch = col.sweep_samples(0)
    fps, n_legs = mean_flops_per_sample(prob, col)
    sweeps_per_step = 2 if method == "heun" else 1
    logf = torch.tensor(np.log(f0), dtype=torch.float64, device="cuda").contiguous()
    t = torch.full((1,), T0, dtype=torch.float64, device="cuda")
    dt = torch.full((1,), DT, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # warm-up steps train the maps (and the budgets); the launch shape is
        # then tuned on the trained state, which the timed steps resemble (the
        # autotuner restores the state after its trial sweeps), and one more
        # untimed step captures the step graph with the chosen kernel
        col.evolve(logf, t, dt, args.warmup, DT, method, stream=stream)
        torch.cuda.synchronize()
        ctas_per_sm = col.autotune(torch.exp(logf), float(t.item()))
        shape = col.launch_shape()
        col.profile(True)
        col.evolve(logf, t, dt, 1, DT, method, stream=stream)
        col.check(stream)
        clocks = Clocks(dev)
        torch.cuda.synchronize()
        barrier()
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launches = 0
        for _ in range(args.steps):
            col.evolve(logf, t, dt, 1, DT, method, stream=stream)
            launches += col.last_launch_count()
            flush.zero_()                                  # evict L2 between steps
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        kern_ms, kern_n = col.profile_read()               # launches of the last timed step
        col.profile(False)
        col.check(stream)
        if VARB:
            # variance-driven budgets: the per-sweep samples as the timed steps set them
            evals = col.sweep_samples()
            samples_per_launch = col.sweep_samples(0)
    from paper_2603_28848_gb300.dist import aggregate
    ms, sweeps = aggregate(ms, sweeps_per_step * args.steps, device="cuda")   # max time, summed units
    sweeps_per_s = sweeps / (ms / 1e3)
    med32, max32 = rel_err_stats(col)

    # ---------------- e2e: host buffers through the public API --------------------------
    h_logf = torch.tensor(np.log(f0), dtype=torch.float64).pin_memory()
    h_t = torch.full((1,), T0, dtype=torch.float64).pin_memory()
    h_out = torch.empty_like(h_logf).pin_memory()
    h_tout = torch.empty_like(h_t).pin_memory()
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        barrier()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(args.steps):
            logf.copy_(h_logf, non_blocking=True)
            t.copy_(h_t, non_blocking=True)
            col.evolve(logf, t, dt, 1, DT, method, stream=stream)
            h_out.copy_(logf, non_blocking=True)
            h_tout.copy_(t, non_blocking=True)
            flush.zero_()
        e3.record(stream)
        torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3)
    ms_e2e, _ = aggregate(ms_e2e, 0, device="cuda")
    vjp = None
    if WORKLOAD_KEY == "c5" or args.vjp:
        v = torch.ones_like(logf)
        fcur = torch.exp(logf)
        col.vjp(fcur, v, float(t.item()))
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record()
        for _ in range(3):
            col.vjp(fcur, v, float(t.item()))
        b1.record()
        torch.cuda.synchronize()
        vms = b0.elapsed_time(b1) / 3
        vjp = {"ms_per_vjp": vms, "samples": col.sweep_samples(0),
               "samples_per_s": col.sweep_samples(0) / (vms / 1e3),
               "what": "dL/df, dL/dm, dL/dcoupling of v.C~ (fixed samples, one iteration per task), FP32"}
    implicit = None
    if WORKLOAD_KEY == "c5" or args.implicit:
        fcur = torch.exp(logf)
        tt = float(t.item())
        u = fcur.clone()
        C, _ = col.jvp(fcur, u, tt)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record()
        for _ in range(3):
            col.jvp(fcur, u, tt)
        b1.record()
        torch.cuda.synchronize()
        jms = b0.elapsed_time(b1) / 3
        rate = float((C / fcur).abs().max().item())
        dt_imp = 10.0 * prob.eps_dt / rate           # ten times the explicit bound of Eq. (16)
        lg = logf.clone()
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        info = col.step_implicit_euler(lg, tt, dt_imp, train=False, max_newton=12, krylov_dim=32,
                                       raise_on_failure=False)
        ims = (time.perf_counter() - c0) * 1e3
        implicit = {"ms_per_jvp": jms, "ms_per_step": ims, "dt": dt_imp, "dt_over_explicit_bound": 10.0, **info,
                    "what": "backward Euler of log f, Newton-GMRES on the fixed-sample C~ (maps kept), FP32"}
    col.close()

    # ---------------- FP64 path (same workload, fewer steps) ---------------------------------
    fp64 = None
    if not args.skip_fp64:
        col64 = Collision(prob, W.PREC_FP64)
        logf64 = torch.tensor(np.log(f0), dtype=torch.float64, device="cuda").contiguous()
        t64 = torch.full((1,), T0, dtype=torch.float64, device="cuda")
        dt64 = torch.full((1,), DT, dtype=torch.float64, device="cuda")
        f64 = torch.exp(logf64)
        col64.eval(f64, T0)                           # warm-up sweep (maps adapt)
        torch.cuda.synchronize()
        col64.profile(True)
        s64 = torch.cuda.current_stream()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s64)
        for _ in range(args.fp64_steps):
            dt64.fill_(DT)
            (col64.step_heun if method == "heun" else col64.step_euler)(logf64, t64, dt64)
        a1.record(s64)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1)
        k64_ms, k64_n = col64.profile_read()
        col64.check()
        med64, max64 = rel_err_stats(col64)
        s64 = sweeps_per_step * args.fp64_steps / (ms64 / 1e3)
        fp64 = {"sweeps_per_s": s64, "evals_per_s": s64 * evals,
                "sweeps_per_s_at_1e-4": s64 / (med64 / 1e-4) ** 2,
                "rel_err_median": med64, "rel_err_max": max64, "steps": args.fp64_steps, "warmup_sweeps": 1,
                "sample_kernel_ms_per_launch": k64_ms / max(k64_n, 1)}
        col64.close()

    # ---------------- roofline of the dominant kernel ----------------------------------------
    per_launch_ms = kern_ms / max(kern_n, 1)
    flops = fps * samples_per_launch
    achieved = flops / (per_launch_ms / 1e3) / 1e12
    peaks = measured_peaks()
    peak = FP32_PEAK_TFLOPS_NOMINAL
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": TRAFFIC_BYTES_PER_LAUNCH,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the sample kernel "
                              "(profiles/eval_kernel_f32_c2_bose_2to2.md); the tables it reads do not "
                              "grow with the sample count",
            "kernel": f"best::eval_kernel<float,{max(n_legs, 4)},{ctas_per_sm},_,{shape[1]},{shape[2]}> (persistent "
                      "sample kernel)",
            "flops_per_sample": fps,
            "samples_per_launch": samples_per_launch, "launch_ms": per_launch_ms,
            "share_of_step": kern_ms / (ms / args.steps) if ms > 0 else None,
            "peak_basis": "152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz max SM clock (nominal unit "
                          "counts; MEASURED_PEAKS.json has no FP32 figure)"}
    if WORKLOAD_KEY == "c2":
        issued = INSTR_PER_SAMPLE_C2 * samples_per_launch / (per_launch_ms / 1e3) / 1e12
        roof["issue"] = {"achieved": issued, "peak": ISSUE_PEAK_TINSTR, "unit": "T thread-instructions/s",
                         "frac": issued / ISSUE_PEAK_TINSTR, "instructions_per_sample": INSTR_PER_SAMPLE_C2,
                         "source": "ncu capture in profiles/eval_kernel_f32_c2_bose_2to2.md"}
        roof["flops_per_sample_ncu"] = MEASURED_FLOPS_PER_SAMPLE_C2

    out = {
        "metric": METRIC, "value": sweeps_per_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; BE(T=1) + Gaussian bump, no dataset)",
        "config": {"workload": f"{wl[0]}: {wl[4]}" + (" + stratified sampling (VEGAS+)" if STRAT else "")
                   + (" + variance-driven budgets" if VARB else ""),
                   "grid_points": prob.grid.n, "tasks": col_tasks, "neval": prob.processes[0].neval,
                   "nitn": prob.processes[0].nitn,
                   "step": f"one {method} step = {sweeps_per_step} sweep(s)", "l2": "flushed between steps "
                   "(512 MiB write, in the timed region)", "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "evals_per_s": sweeps_per_s * evals,
        "evals_per_sweep": evals,
        "sweeps_per_s_at_1e-4": sweeps_per_s / (med32 / 1e-4) ** 2,
        "rel_err_median": med32, "rel_err_max": max32,
        "fp64": fp64,
        "fp32_over_fp64_at_1e-4": (sweeps_per_s / world / (med32 / 1e-4) ** 2) / fp64["sweeps_per_s_at_1e-4"]
        if fp64 else None,
        "roofline": roof,
        "vjp": vjp,
        "implicit_euler": implicit,
        "e2e": {"value": sweeps / (ms_e2e / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": logf.numel() * 8 + 8, "d2h_bytes_per_step": logf.numel() * 8 + 8},
        "graph": "Heun steps replayed from a CUDA graph (best_evolve)",
        "autotune_ctas_per_sm": ctas_per_sm,
        "autotune_shape": dict(zip(("ctas_per_sm", "threads", "samples_per_lane"), shape)),
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.skip_cpu:
        out["fp32_parity"] = fp32_parity(prob, workload()[1], T0)
    if rank == 0 and not args.skip_cpu and WORKLOAD_KEY == "c2":
        with oracle_pool() as pool:
            out["cpu_baseline"] = cpu_baseline(prob, workload()[1], args.cpu_seconds, evals, pool)
    return out


def point_costs(prob):
    """Per grid point: samples x (dimensions + 6) summed over its tasks (the
    sample kernel's cost model), for balancing grid-point shards."""
    n = prob.grid.n
    cost = np.zeros(n)
    for p in prob.processes:
        legs = len(p.species_in) + len(p.species_out)
        sym = sorted(p.species_in) == sorted(p.species_out)
        sides = len(set(p.species_in)) + (0 if sym else len(set(p.species_out)))
        per = np.asarray(p.neval_per_point if p.neval_per_point is not None else [p.neval] * n, dtype=np.float64)
        cost += 2 * sides * per * (3 * (legs - 2) + 6)
    return cost


def run_sharded(args, rank, world):
    """The paper's decomposition over ranks (Sec. 3D, Eq. (17)): one workload,
    rank r evaluating the tasks of a contiguous, cost-balanced block of grid
    points; one NCCL all-reduce of C per evaluation; every rank applies the
    same step stages (strong scaling: the whole job is fixed as N grows)."""
    import torch

    import workloads as W
    from paper_2603_28848_gb300 import Collision, build
    from paper_2603_28848_gb300 import dist as bdist

    build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    prob, f0 = workload()
    wl = WORKLOADS[WORKLOAD_KEY]
    method, DT, T0 = wl[1], wl[2], wl[3]
    lo, hi = bdist.shard(point_costs(prob), rank, world)
    col = Collision(prob, W.PREC_FP32, points=(lo, hi))
    logf = torch.tensor(np.log(f0), dtype=torch.float64, device="cuda").contiguous()
    t = torch.full((1,), T0, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctas_per_sm = col.autotune(torch.exp(logf), T0)
    ref = torch.cuda.Event(enable_timing=True)
    ref.record()

    def clock():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        e.synchronize()
        return ref.elapsed_time(e)

    barrier = torch.distributed.barrier
    clocks = Clocks(dev)
    clocks.start()
    col.profile(True)
    ms, sweeps = bdist.timed_sharded_steps(col, logf, t, dt, DT, method, args.steps, args.warmup, clock, barrier)
    kern_ms, kern_n = col.profile_read()
    col.profile(False)
    clk = clocks.stop()
    col.check()
    tm = torch.tensor([ms], dtype=torch.float64, device="cuda")
    torch.distributed.all_reduce(tm, op=torch.distributed.ReduceOp.MAX)
    ms = float(tm.item())
    # end to end: the step's distribution from pinned host memory and back
    h_logf = torch.tensor(np.log(f0), dtype=torch.float64).pin_memory()
    h_out = torch.empty_like(h_logf).pin_memory()

    def e2e_reduce(x):
        return bdist.all_reduce_sum(x)

    barrier()
    e0 = clock()
    for _ in range(args.steps):
        logf.copy_(h_logf, non_blocking=True)
        bdist.sharded_step(col, logf, t, dt, DT, method, reduce=e2e_reduce)
        h_out.copy_(logf, non_blocking=True)
    e1 = clock()
    barrier()
    te = torch.tensor([e1 - e0], dtype=torch.float64, device="cuda")
    torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
    ev = torch.tensor([float(col.sweep_samples())], dtype=torch.float64, device="cuda")
    torch.distributed.all_reduce(ev)                     # the shards' samples add up to one whole sweep
    evals = float(ev.item())
    per_launch_ms = kern_ms / max(kern_n, 1)
    out = {
        "metric": METRIC, "value": sweeps / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; no dataset)",
        "config": {"workload": f"{wl[0]}: {wl[4]}", "grid_points": prob.grid.n,
                   "step": f"one {method} step = {2 if method == 'heun' else 1} sweep(s) of the whole grid",
                   "parallelism": f"grid points sharded over {world} ranks, one all-reduce of C per evaluation",
                   "shard_of_rank0": [lo, hi] if rank == 0 else None,
                   "l2": "inputs and maps per task are small; no flush (a host round trip per stage)"},
        "sample_kernel_ms_per_launch_rank0": per_launch_ms,
        "autotune_ctas_per_sm": ctas_per_sm,
        "gpu_launches": None,
        "e2e": {"value": sweeps / (float(te.item()) / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": logf.numel() * 8, "d2h_bytes_per_step": logf.numel() * 8},
        "clocks": clk,
        "evals_per_sweep": evals,
        "evals_per_s": evals * sweeps / (ms / 1e3),
    }
    col.close()
    return out


def _oracle_tasks(prob, f0, seconds, first=0):
    """Whole oracle tasks (all iterations, reduced budget) for `seconds`;
    returns (samples evaluated, elapsed s, tasks)."""
    from dataclasses import replace

    from oracle import collision as ocol
    from oracle import vegas
    from oracle.tasks import side_integrals

    small = replace(prob, processes=tuple(replace(p, neval=CPU_NEVAL) for p in prob.processes))
    sis = side_integrals(small)
    dists = ocol.distributions(small, f0, 0.0)
    pts = [5, 40, 70, 100, 120, 20, 60, 90]
    t0 = time.perf_counter()
    done = 0
    k = first
    while time.perf_counter() - t0 < seconds:
        si_idx = k % len(sis)
        i = pts[(k // len(sis)) % len(pts)] % prob.grid.n
        term = k % 2
        si = sis[si_idx]
        p = small.processes[si.process]
        ocol.evaluate_task(small, si_idx, si, i, term, f0, 0.0, vegas.uniform_edges(si.dim, p.nbins), 0,
                           "f32", dists)
        done += CPU_NEVAL * p.nitn
        k += 1
    return done, time.perf_counter() - t0, k - first


def _oracle_worker(job):
    prob, f0, seconds, first = job
    return _oracle_tasks(prob, f0, seconds, first)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(prob, f0, seconds, evals, pool=None, single=True):
    """The oracle, as it stands, on a bounded sample of the same workload:
    whole tasks (all iterations) at a reduced budget, scaled by evals; on
    one core, and (with a spawn pool) on every host core at once, each
    worker running its own tasks for the same time."""
    out = None
    if single or pool is None:
        done, el, k = _oracle_tasks(prob, f0, seconds)
        evs1 = done / el
        out = {"value": evs1 / evals, "unit": UNIT, "cores": 1, "kind": "oracle", "evals_per_s": evs1,
               "sample": f"{k} whole tasks ({prob.processes[0].nitn} iterations, {CPU_NEVAL} samples each) of "
                         f"the same workload, {el:.1f} s on one core; sweeps/s = oracle evals/s / evals per "
                         f"sweep ({evals:.3g})"}
    if pool is not None:
        n = host_cores()
        res = pool.map(_oracle_worker, [(prob, f0, seconds, 1000 * w) for w in range(n)])
        evs = sum(d / e for d, e, _ in res)
        out = {"value": evs / evals, "unit": UNIT, "cores": n, "kind": "oracle", "evals_per_s": evs,
               "sample": f"{sum(r[2] for r in res)} whole tasks ({prob.processes[0].nitn} iterations, {CPU_NEVAL} "
                         f"samples each) of the same workload in {n} concurrent processes, {seconds:.1f} s each; "
                         f"evals/s summed over the processes; sweeps/s = evals/s / evals per sweep ({evals:.3g})",
               "single_core": out}
    return out


PARITY_TASKS = 24   # tasks of the FP32-vs-oracle check in the CPU-baseline leg


def fp32_parity(prob, f0, t):
    """FP32 rounding of the sample kernel on this workload: one iteration from
    uniform maps at the oracle's reduced budget (CPU_NEVAL samples per task),
    so that the FP32 kernel and the oracle (FP64 arithmetic on the same
    FP32-form uniforms) see identical samples and differ by rounding only.
    PARITY_TASKS tasks spread over side integrals, grid points and terms;
    tasks below 1e-8 of the largest checked value of their side integral and
    term are left out (FP32 underflow of negligible tasks).  Runs with the
    CPU baseline (the oracle executes on the host)."""
    import torch

    import workloads as W
    from oracle import collision as ocol
    from oracle import vegas
    from oracle.tasks import side_integrals

    from paper_2603_28848_gb300 import Collision
    one = prob.with_budget(neval=CPU_NEVAL, nitn=1)
    col = Collision(one, W.PREC_FP32)
    try:
        col.eval(torch.tensor(np.ascontiguousarray(f0), dtype=torch.float64, device="cuda"), t)
        col.check()
        mean, _ = col.task_results()
    finally:
        col.close()
    sis = side_integrals(one)
    dists = ocol.distributions(one, f0, t)
    n = one.grid.n
    rows = []
    for k in range(PARITY_TASKS):
        si_idx = k % len(sis)
        term = (k // len(sis)) % 2
        i = (7 + 37 * k) % n
        si = sis[si_idx]
        p = one.processes[si.process]
        om = ocol.evaluate_task(one, si_idx, si, i, term, f0, t, vegas.uniform_edges(si.dim, p.nbins), 0, "f32",
                                dists)[0]
        rows.append((si_idx, term, om, mean[(si_idx * n + i) * 2 + term]))
    big = {}
    for si_idx, term, om, _ in rows:
        big[(si_idx, term)] = max(big.get((si_idx, term), 0.0), abs(om))
    rel = [abs(g - om) / abs(om) for si_idx, term, om, g in rows if om != 0 and abs(om) > 1e-8 * big[(si_idx, term)]]
    return {"tasks": len(rel), "max_rel": float(max(rel)) if rel else None,
            "median_rel": float(np.median(rel)) if rel else None,
            "what": f"FP32 sample kernel vs the FP64 oracle on identical samples (one iteration, uniform maps, "
                    f"{CPU_NEVAL} samples per task): relative difference of the task estimates"}


def oracle_pool():
    """A spawn pool over the host cores (spawn: safe after CUDA use)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(host_cores())


def run_reference(args, rank, world):
    """The oracle timed on the host cores (the reference arm: there is no other
    implementation of the paper's method to run)."""
    prob, _ = workload()
    # evaluations per sweep: 2 species x 128 points x (gain, loss) x nitn x neval
    evals = sum(2 * prob.grid.n * p.nitn * p.neval for p in prob.processes)
    f0 = workload()[1]
    vals = []
    walls = []
    with oracle_pool() as pool:
        for _ in range(args.warmup):
            cpu_baseline(prob, f0, 1.0, evals, pool, single=False)
        for k in range(args.steps):
            w0 = time.perf_counter()
            vals.append(cpu_baseline(prob, f0, args.ref_seconds, evals, pool, single=k == args.steps - 1))
            walls.append(time.perf_counter() - w0)
    v = statistics.mean(b["value"] for b in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    samples = [b["evals_per_s"] * args.ref_seconds for b in vals]
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            # wall time of one timed step as it ran (a bounded sample of the workload, on every host core)
            "ms_per_step": 1e3 * statistics.mean(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "arm": f"CPU oracle, {cb['cores']} host cores"},
            "timed": {"steps": args.steps, "seconds_per_step": statistics.mean(walls),
                      "samples_per_step": statistics.mean(samples), "samples_per_task_iteration": CPU_NEVAL,
                      "note": "each step runs whole oracle tasks at a reduced budget for a fixed time; value "
                              "(sweeps/s) is extrapolated: evals/s divided by the evaluations of one full sweep; "
                              f"one full sweep would take {1e3 / v if v > 0 else float('nan'):.4g} ms"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--neval", type=int, default=None,
                    help="samples per task per iteration (smaller cases for profiling)")
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--vjp", action="store_true", help="also time the adjoint")
    ap.add_argument("--implicit", action="store_true", help="also time the tangent and one implicit Euler step")
    ap.add_argument("--strat", action="store_true", help="adaptive stratified sampling (VEGAS+) in every process")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: an independent replica per rank instead of the grid-point shards")
    ap.add_argument("--variance-budgets", action="store_true",
                    help="multi-species workload: per-task budgets re-set from the last sweep's variance")
    args = ap.parse_args()
    global NEVAL, WORKLOAD_KEY, STRAT, VARB
    VARB = args.variance_budgets
    NEVAL = args.neval
    STRAT = args.strat
    WORKLOAD_KEY = args.workload
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        os.environ.setdefault("NCCL_DEBUG", "INFO")          # communicator lines name the ranks of the run
        os.environ.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    out = run_sharded(args, rank, world) if world > 1 and not args.replicas else run_native(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
