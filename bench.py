"""Benchmark: space-time DoF/s of the monolithic Biot slab march on one GB300.

Workload (one "step", the precision configuration): 3-D Biot on the unit cube,
64^3 hexes, Q2 / RT1 / DGQ1, dG(2) in time, T = 1 in 8 slabs (44.6 M unknowns per
slab; `--n 32 --r 1 --slabs 16` gives the 32^3 dG(1) workload); layered log-normal permeability
K = exp(g) 1e-2 (g ~ N(0, 1.5^2) per 4-cell z-layer, seed 1801); lambda = mu = 1,
b = 0.8, 1/M = 0.05; unit compressive load on the drained top face, roller /
no-flow elsewhere.  Every slab is solved to relative residual 1e-10 (FP64) by
the mixed FP32-inner / FP64-refinement solver (the metric's headline) and, for
comparison, by the all-FP64 solver; the relative difference of the two end
states is reported.

value = N_slab * slabs / (device time of one mixed-precision march).
e2e   = the same metric through the C ABI with host buffers (the load vector,
        the initial state and the end state copied inside the timed region).

`--impl reference` times the FP64 CPU oracle (sparse direct solves) on a
bounded sample of the same problem class instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "slab solve time & space-time DoF/s at 1e-8 rel err: mixed-precision vs FP64, 1 GB300"
WORKLOAD = ("3D Biot, unit cube, {n}^3 hexes, Q2 displacement / RT1 flux / DGQ1 pressure, dG({r}), T=1 in {slabs} slabs; "
            "layered log-normal K (std 1.5, 4-cell z-layers, seed 1801); lambda=mu=1, b=0.8, 1/M=0.05; "
            "drained top with unit compressive load, roller/no-flow elsewhere")
COEF = dict(lam=1.0, mu=1.0, b=0.8, invM=0.05, eta=1.0, K_dr=1.0 + 2.0 / 3.0)


def consolidation_bcs(d):
    ubc = [2] * (2 * d)
    ubc[-1] = 0
    fbc = [1] * (2 * d)
    fbc[-1] = 0
    return ubc, fbc


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summary()

    def summary(self):
        """Median SM clock under load, maximum clock and the throttle reasons seen in the rows."""
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for i, nm in enumerate(names):
                if r[5 + i].lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def hbm_peak_measured(root):
    try:
        return json.load(open(os.path.join(root, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        return 6800.0


def whole_job_rate(units_per_rank, t_local, world_size, device=None):
    """Replica runs: every rank processed units_per_rank in t_local seconds; the job took as
    long as its slowest rank (max over ranks).  Returns (whole-job units/s, job seconds)."""
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    if world_size > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    t_job = float(t.item())
    return world_size * units_per_rank / t_job, t_job


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(seconds_target=15.0, n=4, slabs=16):
    """FP64 CPU oracle (sparse LU) on a bounded sample: 3-D n^3 hexes, same
    coefficients/loading, dG(1), `slabs` slabs; repeated to ~seconds_target."""
    from oracle.slab import SlabProblem
    from oracle.space import Mesh, load_vector
    from paper_1801_04984_gb300.inputs import layered_logk, K0
    m = Mesh((n, n, n))
    g = layered_logk(m.n, layer_cells=max(1, n // 8), std=1.5, seed=1801)
    co = dict(COEF, K=K0 * np.exp(g))
    ubc, fbc = consolidation_bcs(3)

    def trac(X, t, f):
        o = np.zeros((len(X), 3))
        o[:, 2] = -1.0
        return o
    F = load_vector(m, 0.0, traction=trac, u_bc=ubc, f_bc=fbc)
    t0 = time.perf_counter()
    reps = 0
    dofs = 0
    while True:
        prob = SlabProblem(m, co, 1, ubc, fbc)
        prob.march(1.0, slabs, lambda t: F)
        reps += 1
        dofs += prob.Nslab * slabs
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    return {"value": dofs / dt, "unit": "DoF/s", "cores": 1, "kind": "oracle", "seconds": dt,
            "sample": "3-D %d^3 hexes, dG(1), %d slabs, N_slab=%d, x%d marches (assembly + SuperLU factorisation + "
                      "solves), %.1f s" % (n, slabs, prob.Nslab, reps, dt),
            "host_cores": os.cpu_count()}


def profile_figure(name, key):
    """A figure recorded in a committed ncu summary under profiles/ (the line `key value`), or None."""
    try:
        for line in open(os.path.join(ROOT, "profiles", name)).read().splitlines():
            if line.startswith(key):
                return float(line.split(":")[1])
    except (OSError, ValueError):
        pass
    return None


def schur_roofline(sch, weight_bytes_per_launch, t_prof, hbm_peak, traffic_per_unit=None, traffic_file=None):
    """HBM roofline of the flux-pressure Schur Chebyshev step k_schur_cheb_mf<float> from its
    launches in one march, sch = (launches, ms, units), units = pressure point x right-hand side.
    Algorithmic bytes of a step: per point and right-hand side x, b and the previous direction d
    read and the new direction and iterate written (5 x 4 B); per launch the flux weights of the
    instance (one float per flux DoF) read once.  About 45 flop per point and right-hand side
    against those 20+ bytes: far below the FP32 ridge point, so the bound is HBM."""
    n, ms, units = sch
    if n <= 0 or ms <= 0:
        return None
    alg = 20.0 * units + weight_bytes_per_launch * n
    ach = alg / (ms / 1e3) / 1e9
    out = {"bound": "hbm", "kernel": "k_schur_cheb_mf<float> (one matrix-free Chebyshev step of the flux-pressure Schur solve)",
           "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)",
           "traffic": None, "traffic_source": None,
           "launches_per_step": n, "avg_launch_us": 1e3 * ms / n,
           "share_of_step": (ms / 1e3) / t_prof if t_prof > 0 else None,
           "algorithmic_bytes_per_launch": alg / n}
    if traffic_per_unit:
        out["traffic"] = traffic_per_unit * units / n
        out["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of a one-column step (%s), per point x "
                                 "right-hand side, times the average units of one launch of this march" % traffic_file)
    return out


def dominant_roofline(*rooflines):
    """(the roofline object with the largest share of the profiled step, the next one)."""
    ok = [r for r in rooflines if r and r.get("share_of_step")]
    if not ok:
        return (rooflines[0] if rooflines else None), None
    ok.sort(key=lambda r: r["share_of_step"], reverse=True)
    return ok[0], (ok[1] if len(ok) > 1 else None)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    per = []
    for _ in range(args.warmup + args.steps):
        per.append(oracle_sample(seconds_target=max(2.0, 20.0 / (args.steps + args.warmup)), n=4, slabs=16))
    timed = per[args.warmup:]
    val = float(np.mean([p["value"] for p in timed]))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean([p["seconds"] for p in timed])), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(n=args.n, r=args.r, slabs=args.slabs),
                       "measured_on": "a bounded sample of this problem class on the host cores (see cpu_baseline.sample)"},
            "cpu_baseline": {"value": val, "unit": "DoF/s", "cores": 1, "kind": "oracle", "sample": timed[0]["sample"]},
            "e2e": {"value": val, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """256 independent 2-D instances (n in {16,32,64,128}, r in {0,1,2}, correlated log-normal K
    with std 1.0 and 8-cell correlation, 4 slabs, unit top load), FP32 inner / FP64 refinement
    to relative residual 1e-8, solved by biot_solve_batch.  value = total space-time DoF / s."""
    import torch
    torch.cuda.set_device(0)
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import batch_instances, correlated_logk_2d, K0
    ubc, fbc = consolidation_bcs(2)
    desc = batch_instances(args.instances, seed=1801)
    inst = []
    dofs = 0
    for d in desc:
        n, r = d["n"], d["r"]
        K = K0 * np.exp(correlated_logk_2d(n, std=1.0, corr_cells=8.0, seed=d["seed"]))
        nu = (2 * n + 1) ** 2
        n_space = 2 * nu + 2 * (2 * n + 1) * (2 * n) + (2 * n) ** 2
        dofs += n_space * (r + 1) * 4
        inst.append(dict(dim=2, n=(n, n), coeffs=dict(COEF, K=K), r=r, T=1.0, slabs=4, u_bc=ubc, f_bc=fbc,
                         load_kind=B.LOAD_TRACTION_TOP, load_value=1.0, U_end=np.zeros(n_space)))
    times = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, status, stats = B.solve_batch(inst, workers=args.workers, tol=args.batch_tol, mode=B.MIXED,
                                          opts=dict(schur_mg=args.schur_mg) if args.schur_mg else None)
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
        assert rc == 0, (rc, [s for s in status if s])
    t = float(np.mean(times))
    iters = [s["iterations"] for s in stats]
    # relative error of the mixed end states against FP64 marches (relative residual 1e-12) on
    # a seeded sample of 8 instances, one per 32 (every (n, r) mix is represented)
    errs = []
    for i in range(0, len(inst), max(1, len(inst) // 8)):
        ref = dict(inst[i], U_end=np.zeros_like(inst[i]["U_end"]))
        rc_ref, _, _ = B.solve_batch([ref], workers=1, tol=1e-12, mode=B.FP64, max_iters=20000)
        assert rc_ref == 0, rc_ref
        errs.append(float(np.linalg.norm(inst[i]["U_end"] - ref["U_end"]) / np.linalg.norm(ref["U_end"])))
    line = {"metric": METRIC + " (batching workload)", "value": dofs / t, "unit": "DoF/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "%d independent 2-D Biot instances, n in {16,32,64,128}, dG(r) r in {0,1,2}, "
                                   "correlated log-normal K (std 1.0, 8-cell correlation), 4 slabs each, "
                                   "FP32 inner + FP64 refinement to relative residual %g; instances of equal (n, r) solved as one batched "
                                   "context (all instances in every launch)" % (args.instances, args.batch_tol),
                       "instances_per_s": args.instances / t, "total_space_time_dofs": dofs,
                       "mean_iterations_per_instance": float(np.mean(iters))},
            "error_vs_fp64": {"max": max(errs), "instances_checked": len(errs),
                              "definition": "||U_end(mixed, residual tol) - U_end(FP64, residual 1e-12)|| / ||U_end(FP64)||"}}
    print(json.dumps(line), flush=True)
    return 0


def run_apply(args):
    """One slab-operator apply (FP64 and FP32) of the layered 3-D problem at n^3, dG(r), timed
    with CUDA events (median of `steps`, L2 flushed before each), against the HBM roofline:
    algorithmic bytes = read x + write y + one coefficient per cell, (2 N_slab + cells) x word."""
    import torch
    torch.cuda.set_device(0)
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import layered_logk, K0
    n, r = args.n, args.r
    g = layered_logk((n, n, n), layer_cells=4, std=1.5, seed=1801)
    ubc, fbc = consolidation_bcs(3)
    ctx = B.Context(3, (n, n, n), dict(COEF, K=K0 * np.exp(g)), r, ubc, fbc)
    tau = 1.0 / args.slabs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"config": {"workload": "one slab-operator apply: " + WORKLOAD.format(n=n, r=r, slabs=args.slabs),
                      "n_slab": ctx.n_slab, "l2": "256 MB buffer written before every timed apply"}}
    for dt, name in ((torch.float64, "fp64"), (torch.float32, "fp32")):
        x = torch.randn(ctx.n_slab, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(max(1, args.warmup)):
            ctx.apply_slab(tau, x, y)
        ts = []
        for _ in range(max(1, args.steps)):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            ctx.apply_slab(tau, x, y)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = float(np.median(ts))
        algo = (2 * ctx.n_slab + ctx.n_cells) * x.element_size()
        out[name] = {"ms": t * 1e3, "algorithmic_MB": algo / 1e6, "achieved_GBs": algo / t / 1e9,
                     "hbm_peak_GBs": hbm_peak_measured(ROOT), "frac_of_hbm": algo / t / 1e9 / hbm_peak_measured(ROOT),
                     "slab_dofs_per_s": ctx.n_slab / t}
    ctx.destroy()
    print(json.dumps(out), flush=True)
    return 0


def run_kernels(args):
    """Per-kernel timings of the operator pieces on the layered 3-D problem at n^3, dG(r), without
    a solve (no Krylov bases: a few GB on the device): the FP32 elasticity operator on one column,
    one FP32 multigrid V-cycle, one FP32 flux-pressure Schur Chebyshev step, and FP32 / FP64 slab
    applies; CUDA events, median of `steps`, L2 flushed before each.  One more V-cycle and Schur
    step run inside the NVTX ranges 'vcycle' and 'schur_step' (for single-kernel profiler
    captures)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import layered_logk, K0
    n, r = args.n, args.r
    g = layered_logk((n, n, n), layer_cells=4, std=1.5, seed=1801)
    ubc, fbc = consolidation_bcs(3)
    ctx = B.Context(3, (n, n, n), dict(COEF, K=K0 * np.exp(g)), r, ubc, fbc)
    tau = 1.0 / args.slabs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(1801)
    xs = torch.rand(ctx.n_space, device="cuda", generator=gen) - 0.5
    ys = torch.empty_like(xs)
    xl = torch.rand(ctx.n_slab, device="cuda", generator=gen) - 0.5
    yl = torch.empty_like(xl)
    xl64, yl64 = xl.double(), torch.empty(ctx.n_slab, dtype=torch.float64, device="cuda")

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        ts = []
        for _ in range(max(1, args.steps)):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return float(np.median(ts))
    out = {"metric": "operator kernel timings (us, CUDA events, median)", "n_gpus": 1, "dtype": "f32/f64",
           "data": "synthetic", "config": {"workload": "kernels of: " + WORKLOAD.format(n=n, r=r, slabs=args.slabs),
                                           "l2": "256 MB buffer written before every timed call"}}
    peak32, _ = B.fma_peak(B.FP32)
    ctx.profile(True)
    ctx.kernel_stats(B.KERNEL_ELASTICITY_FP32)
    t1 = timed(lambda: ctx.apply_part(B.PART_ELASTICITY, tau, xs, ys))
    k1 = ctx.kernel_stats(B.KERNEL_ELASTICITY_FP32)
    ctx.profile(False)
    nodes = (2 * n + 1) ** 3
    out["elasticity_fp32_1col_us"] = t1
    out["elasticity_fp32_1col_kernel_us"] = 1e3 * k1[1] / max(1, k1[0])
    out["elasticity_fp32_1col_frac_of_fp32_peak"] = 360.0 * nodes / (k1[1] / max(1, k1[0]) / 1e3) / 1e12 / peak32
    out["vcycle_fp32_us"] = timed(lambda: ctx.apply_part(B.PART_VCYCLE, tau, xs, ys))
    out["schur_step_fp32_us"] = timed(lambda: ctx.apply_part(B.PART_SCHUR_STEP, tau, xs, ys))
    out["slab_apply_fp32_us"] = timed(lambda: ctx.apply_slab(tau, xl, yl))
    out["slab_apply_fp64_us"] = timed(lambda: ctx.apply_slab(tau, xl64, yl64))
    out["fp32_fma_peak_tflops"] = peak32
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("vcycle")
    ctx.apply_part(B.PART_VCYCLE, tau, xs, ys)
    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("schur_step")
    ctx.apply_part(B.PART_SCHUR_STEP, tau, xs, ys)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ctx.destroy()
    print(json.dumps(out), flush=True)
    return 0


def run_dwr(args):
    """Goal-oriented time-error estimate of the layered 3-D march (dG(r) against dG(r+1),
    J = mean pressure over [0.4, 0.6]^3 at T^-), mixed precision; device time of the
    whole estimate (forward dG(r) march, backward dG(r+1) dual march, slab residuals)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import layered_logk, K0
    n, r, slabs = args.n, args.r, args.slabs
    g = layered_logk((n, n, n), layer_cells=4, std=1.5, seed=1801)
    ubc, fbc = consolidation_bcs(3)
    co = dict(COEF, K=K0 * np.exp(g))
    ctx = B.Context(3, (n, n, n), co, r, ubc, fbc)
    ctx1 = B.Context(3, (n, n, n), co, r + 1, ubc, fbc)
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    j = torch.zeros_like(f)
    ctx.goal_mean_pressure([0.4] * 3, [0.6] * 3, j)
    U0 = torch.zeros_like(f)
    times = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eta, eta_s, J = ctx.dwr_time_estimate(ctx1, 1.0, slabs, [f], [[1, 0, 0, 0]], U0, j, tol=1e-10, mode=B.MIXED)
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    line = {"metric": "goal-oriented time-error estimate (dual-weighted residual, dG(r) against dG(r+1))",
            "value": t, "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(n=n, r=r, slabs=slabs) + "; J = mean p over [0.4,0.6]^3 at T^-"},
            "J": J, "eta": eta, "eta_per_slab": eta_s}
    print(json.dumps(line), flush=True)
    return 0


def run_fixed_stress(args):
    """The layered 3-D march solved by fixed-stress iterative coupling (FP64 sweeps) and by the
    monolithic FP64 FGMRES, each slab to relative residual 1e-10: DoF/s and sweeps or
    iterations per slab (device time of one march each)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import layered_logk, K0
    n, r, slabs = args.n, args.r, args.slabs
    g = layered_logk((n, n, n), layer_cells=4, std=1.5, seed=1801)
    ubc, fbc = consolidation_bcs(3)
    ctx = B.Context(3, (n, n, n), dict(COEF, K=K0 * np.exp(g)), r, ubc, fbc)
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    U0 = torch.zeros_like(f)
    out = {"metric": "space-time DoF/s of the march: fixed-stress iterative coupling vs monolithic FGMRES (FP64)",
           "unit": "DoF/s", "higher_is_better": True, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD.format(n=n, r=r, slabs=slabs), "tol": 1e-10}}
    for name, mode in (("fixed_stress", B.FIXED_STRESS), ("monolithic_fgmres", B.FP64)):
        U = torch.zeros_like(f)
        ctx.march(1.0, slabs, [f], [[1, 0, 0, 0]], U0, U, tol=1e-10, mode=mode, max_iters=20000)  # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        st = ctx.march(1.0, slabs, [f], [[1, 0, 0, 0]], U0, U, tol=1e-10, mode=mode, max_iters=20000)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[name] = {"value": ctx.n_slab * slabs / t, "ms_per_slab": 1e3 * t / slabs, "iters_per_slab": st["iters_per_slab"],
                     "rel_residual": st["rel_residual"]}
    out["value"] = out["fixed_stress"]["value"]
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--r", type=int, default=2)
    ap.add_argument("--slabs", type=int, default=8)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison march")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer run")
    ap.add_argument("--no-profile", action="store_true",
                    help="skip the extra per-kernel-event step and the FMA peaks (for profiler launch lists)")
    ap.add_argument("--config", default="march", choices=["march", "batch", "apply", "dwr", "fixed_stress", "kernels"],
                    help="march: the layered 3-D march (default 64^3 dG(2), 8 slabs); batch: 256 ragged 2-D instances; "
                         "apply: one slab-operator apply against the HBM roofline; "
                         "dwr: goal-oriented time-error estimate; fixed_stress: iterative coupling vs monolithic; "
                         "kernels: operator-kernel timings without a solve")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--batch-tol", type=float, default=1e-10,
                    help="batch: relative residual of every slab solve (the end states are checked against FP64)")
    ap.add_argument("--workers", type=int, default=0, help="batch: max instances per batched context (0: library default)")
    ap.add_argument("--cheb-degree", type=int, default=0, help="elasticity smoother degree (0: library default)")
    ap.add_argument("--pair-coupling", type=int, default=0, help="0: block Gauss-Seidel on the complex pair, -1: dropped")
    ap.add_argument("--schur-degree", type=int, default=0, help="Schur Chebyshev degree (0: library default)")
    ap.add_argument("--schur-mg", type=int, default=0,
                    help="flow-block Schur solve: 0 library choice, 1 multigrid V-cycle, -1 Chebyshev")
    ap.add_argument("--beta-fs", type=float, default=-1.0,
                    help="fixed-stress parameter of the preconditioner (negative: b^2/K_dr)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "batch":
        return run_batch(args)
    if args.config == "apply":
        return run_apply(args)
    if args.config == "dwr":
        return run_dwr(args)
    if args.config == "fixed_stress":
        return run_fixed_stress(args)
    if args.config == "kernels":
        return run_kernels(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import layered_logk, K0

    n, r, slabs, T = args.n, args.r, args.slabs, 1.0
    g = layered_logk((n, n, n), layer_cells=4, std=1.5, seed=1801)
    ubc, fbc = consolidation_bcs(3)
    ctx = B.Context(3, (n, n, n), dict(COEF, K=K0 * np.exp(g)), r, ubc, fbc,
                    opts=dict(cheb_degree=args.cheb_degree, schur_degree=args.schur_degree,
                              pair_coupling=args.pair_coupling, beta_fs=args.beta_fs, schur_mg=args.schur_mg))
    dev = torch.device("cuda", torch.cuda.current_device())
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device=dev)
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    U0 = torch.zeros_like(f)
    U_mixed = torch.zeros_like(f)
    U_fp64 = torch.zeros_like(f)
    tcoef = [[1.0, 0, 0, 0]]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step(mode, U_end, stats=None):
        s = ctx.march(T, slabs, [f], tcoef, U0, U_end, tol=1e-10, mode=mode)
        if stats is not None:
            stats.append(s)
        return s

    for _ in range(args.warmup):
        step(B.MIXED, U_mixed)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0, _, _ = ctx.counters()
    stats = []
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step(B.MIXED, U_mixed, stats)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    launches1, _, _ = ctx.counters()
    clocks = sampler.stop() if sampler else None
    # one more (untimed) step with CUDA events around every launch of the dominant kernels
    t_prof, el, elc, sch, el64 = 0.0, (0, 0.0, 0.0), (0, 0.0, 0.0), (0, 0.0, 0.0), (0, 0.0, 0.0)
    if not args.no_profile:
        ctx.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step(B.MIXED, U_mixed)
        e1.record(stream)
        torch.cuda.synchronize()
        t_prof = e0.elapsed_time(e1) / 1e3
        el = ctx.kernel_stats(B.KERNEL_ELASTICITY_FP32)
        elc = ctx.kernel_stats(B.KERNEL_ELASTICITY_FP32_COARSE)
        sch = ctx.kernel_stats(B.KERNEL_SCHUR_FP32)
        el64 = ctx.kernel_stats(B.KERNEL_ELASTICITY_FP64)
        ctx.profile(False)
    dofs_step = ctx.n_slab * slabs
    value, t_step = whole_job_rate(dofs_step, float(np.mean(times)), ws, dev)

    # end-to-end through the C ABI with host buffers
    f_host = f.cpu().numpy().copy()
    U0_host = np.zeros(ctx.n_space)
    U_host = np.zeros(ctx.n_space)
    te = []
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.march(T, slabs, [f_host], tcoef, U0_host, U_host, tol=1e-10, mode=B.MIXED)
        torch.cuda.synchronize()
        te.append(time.perf_counter() - t0)
    e2e = None if not te else {"value": ws * dofs_step / float(np.mean(te)), "unit": "DoF/s",
                               "h2d_bytes_per_step": 2 * ctx.n_space * 8, "d2h_bytes_per_step": ctx.n_space * 8}

    # FP64 comparison march (device-timed, outside the headline region)
    fp64 = None
    if not args.no_fp64:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s64 = step(B.FP64, U_fp64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        rel = (torch.linalg.norm(U_mixed - U_fp64) / torch.linalg.norm(U_fp64)).item()
        fp64 = {"value": dofs_step / t64, "unit": "DoF/s", "ms_per_step": t64 * 1e3,
                "ms_per_slab": t64 * 1e3 / slabs, "iterations": s64["iterations"],
                "end_state_rel_diff_mixed_vs_fp64": rel}

    # rooflines of the two dominant kernels; `roofline` is the one with the larger share of the
    # profiled march.  (1) The FP32 elasticity (displacement-row) operator on the fine multigrid
    # levels (the z-marching kernel, grids of >= 1e5 nodes; its launches in one march: smoothing
    # steps, residuals and the slab applies).  Algorithmic work of the
    # sum-factorised Kronecker apply: 180 FMA = 360 flop per Q2 node and right-hand side (z pass
    # 12 outputs x 4 taps, y pass 21 terms x 4, x pass 12 x 4; 5-tap vertex / 3-tap mid rows);
    # algorithmic bytes: the displacement block read once and written once, 3 x 2 x 4 B per node.
    # The kernel is bound by FP32 FMA issue, not HBM: it is reported against the FP32 FMA
    # throughput that biot_fma_peak measures on this GPU in this run.  The FP64 elasticity
    # launches of the same march (the true residuals of the refinement) are reported against
    # the measured FP64 FMA throughput.
    peak32, peak64 = (B.fma_peak(B.FP32)[0], B.fma_peak(B.FP64)[0]) if not args.no_profile else (float("nan"),) * 2
    el_n, el_ms, el_units = el
    achieved = 360.0 * el_units / (el_ms / 1e3) / 1e12 if el_ms > 0 else None
    traffic, traffic_src = None, None
    prof_path = os.path.join(ROOT, "profiles", "elasticity_fp32_%dcube.txt" % n)
    try:
        for line in open(prof_path).read().splitlines():
            if line.startswith("dram_bytes_per_node_rhs:"):
                traffic = float(line.split(":")[1]) * el_units / max(1, el_n)
                traffic_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one fine-level launch (%s), per node "
                               "x right-hand side, times the average units of one launch of this march"
                               % os.path.relpath(prof_path, ROOT))
    except OSError:
        traffic = None
    el_roofline = {"bound": "alu",
                "kernel": "k_elast3_zm (FP32 elasticity operator on the multigrid levels of >= 1e5 nodes)",
                "achieved": achieved, "peak": peak32, "unit": "TFLOP/s",
                "frac": (achieved / peak32) if achieved else None,
                "peak_source": "measured in this run: biot_fma_peak(FP32), independent FMA chains on every SM",
                "traffic": traffic, "traffic_source": traffic_src,
                "launches_per_step": el_n, "avg_launch_us": 1e3 * el_ms / max(1, el_n),
                "share_of_step": (el_ms / 1e3) / t_prof if t_prof > 0 else None,
                "algorithmic_gbs": 24.0 * el_units / (el_ms / 1e3) / 1e9 if el_ms > 0 else None,
                "hbm_peak_gbs": hbm_peak_measured(ROOT)}
    e64_n, e64_ms, e64_units = el64
    ach64 = 360.0 * e64_units / (e64_ms / 1e3) / 1e12 if e64_ms > 0 else None
    fp64_roofline = {"bound": "alu", "kernel": "k_apply_u3_col<double> (FP64 elasticity operator: the true residuals)",
                     "achieved": ach64, "peak": peak64, "unit": "TFLOP/s", "frac": (ach64 / peak64) if ach64 else None,
                     "peak_source": "measured in this run: biot_fma_peak(FP64)",
                     "launches_per_step": e64_n, "avg_launch_us": 1e3 * e64_ms / max(1, e64_n),
                     "share_of_step": (e64_ms / 1e3) / t_prof if t_prof > 0 else None}
    coarse = {"kernel": "k_apply_u3_col<float> (FP32 elasticity operator on the levels below 1e5 nodes)",
              "launches_per_step": elc[0], "avg_launch_us": 1e3 * elc[1] / max(1, elc[0]),
              "share_of_step": (elc[1] / 1e3) / t_prof if t_prof > 0 else None,
              "achieved_tflops": 360.0 * elc[2] / (elc[1] / 1e3) / 1e12 if elc[1] > 0 else None}
    # (2) the flux-pressure Schur Chebyshev step, HBM-bound by its arithmetic intensity
    nqt = ctx.n_space - 3 * (2 * n + 1) ** 3 - 8 * n ** 3  # flux DoFs of one temporal level
    sch_roofline = schur_roofline(sch, 4.0 * nqt, t_prof, hbm_peak_measured(ROOT),
                                  profile_figure("schur_step_fp32_%dcube.txt" % n, "dram_bytes_per_point_rhs:"),
                                  "profiles/schur_step_fp32_%dcube.txt" % n)
    roofline, second = dominant_roofline(el_roofline, sch_roofline)
    s_mean = stats[-1]
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_sample(seconds_target=15.0, n=4, slabs=16)
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(n=n, r=r, slabs=slabs),
                   "n_slab": ctx.n_slab, "slabs": slabs, "solver": "FGMRES(30) FP32 inner + FP64 refinement, tol 1e-10",
                   "l2": "256 MB buffer written before every timed step (> 129 MB L2)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "ms_per_slab": t_step * 1e3 / slabs,
        "iterations_per_step": s_mean["iterations"], "refinements_per_step": s_mean["refinements"],
        "iters_per_slab": s_mean["iters_per_slab"],
        "fp64": fp64,
        "e2e": e2e,
        "gpu_launches": int((launches1 - launches0) / max(1, args.steps)),
        "roofline": roofline,
        "second_kernel": second,
        "coarse_elasticity": coarse,
        "fp64_roofline": fp64_roofline,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
