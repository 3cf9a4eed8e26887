#!/usr/bin/env python
"""Benchmark: PCG time-to-relative-residual 1e-8 on the n = 65536 kernel system.

Workload (one "step"): the ARD-RBF system (K + sigma^2 I) alpha = y with
n = 65536, d = 8, X ~ U[0,1]^8, l_r ~ LogUniform(0.3, 3), s = 1, sigma^2 = 1e-4
(seeded, synthetic), Nystrom preconditioner with m = 1024 random inducing
points built inside the step, solved to ||y - K_y alpha|| <= 1e-8 ||y||
(recomputed in native FP64) by the mixed-precision solver: flexible CG in FP64
(double-float direction products, FP64 certified residuals) around an inner
FP32 PCG with the tensor-core K.V (--precision selects another mode).  Inputs
are resident in HBM when the timed region starts; L2 is flushed between steps.

Printed: one JSON line with the time per solve (seconds, lower is better) on
the production path, the end-to-end time through the C ABI from host buffers,
the roofline of every kernel class (algorithmic work over the pipe rates
measured on this GPU by kpcg_probe_rates), the FP64 CPU oracle's time on a
bounded sample of the same workload, and the same-GPU comparisons (plain FP32
PCG's floor and time to 1e-6, block-Jacobi, the double-float solver).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kpcg|reference]
        [--workload solve65k|batch64|grad45k|warm131k|predict4k|fig1|laplace15k]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402

N_FULL, D, M_INDUCING, TOL = 65536, 8, 1024, 1e-8
METRIC = "PCG time-to-rel-res 1e-8 at n=65k vs plain FP32; K.V TFLOP/s vs roofline"
WORKLOAD = ("ARD-RBF n=65536 d=8 X~U[0,1]^8 l~LogU(0.3,3) s=1 noise=1e-4, y=sum sin(x)+N(0,0.01); "
            "Nystrom m=1024 built in-step; tol 1e-8 rel; 1 RHS")
# The headline solver: flexible CG in FP64 (double-float outer directions,
# native-FP64 certified residuals) around an inner FP32 PCG whose K.V runs on
# the tensor cores, on the operator shifted by inner_shift * sigma^2.  The
# shift and inner tolerance were picked by the sweep that
# `--workload precision` runs.
HEADLINE_PREC = "tc_ir"
MODE_OPTS = {
    "tc_ir": dict(inner_shift=1.0, inner_tol=0.1),
    "fp32_ir": dict(inner_shift=4.0, inner_tol=0.1),
    "xf_ir": dict(inner_shift=0.25, inner_tol=0.3),
    "tcx_ir": dict(inner_shift=0.1, inner_tol=0.5),
    "df64": {},
    "fp64": {},
}


def mode_id(kpcg, name):
    return {"tc_ir": kpcg.KPCG_TC_IR, "fp32_ir": kpcg.KPCG_FP32_IR, "xf_ir": kpcg.KPCG_FP32X_IR,
            "tcx_ir": kpcg.KPCG_TCX_IR, "df64": kpcg.KPCG_DF64, "fp64": kpcg.KPCG_FP64}[name]


def kv_algorithmic(n, d, c):
    """Algorithmic work of one product (K + sigma^2 I) V on n points with c
    columns.  K is symmetric: its n(n+1)/2 distinct entries each need one
    exp2, 2d flops for the squared distance (a difference and an FMA per
    dimension) and, with V, 2c FMAs (row i and, mirrored, column j)."""
    ent = n * (n + 1) / 2.0
    return {"distinct_entries": ent, "ex2": ent, "distance_flops": 2.0 * d * ent,
            "contraction_flops": 2.0 * n * n * c, "fp32_slots": ent * (2 * d + 2 * c)}


def alu_roofline(kernel, n, d, c, ms, rates, fp64=False, tensor_tflops=None):
    """Roofline of one K.V launch of `ms` milliseconds.  frac: the
    tensor/MUFU bound (the exps on the MUFU, the distance and contraction
    flops on the tensor cores at the measured BF16 rate) over the measured
    time, for the n(n+1)/2 distinct entries; frac_simt: the bound with the
    distance and contraction on the FP32 pipe instead (2d + 2c issue slots per
    distinct entry); frac_evaluated: the tensor/MUFU bound for all n^2 entries
    (what a kernel that does not use the symmetry must evaluate).  fp64: the
    native-FP64 residual kernel against the measured FP64 FMA rate (distance,
    contraction and the exp counted as one operation each)."""
    w = kv_algorithmic(n, d, c)
    t = ms / 1e3
    if fp64:
        ops = w["fp32_slots"] + w["ex2"]
        r = rates["fp64_fma_per_s"]
        return {"bound": "alu", "pipe": "fp64", "kernel": kernel, "achieved": ops / t / 1e12,
                "peak": r / 1e12, "unit": "Top/s", "frac": ops / r / t, "avg_ms": ms,
                "algorithmic": w}
    return roofline_from_work(kernel, w, ms, rates, tensor_tflops)


def roofline_from_work(kernel, w, ms, rates, tensor_tflops=None):
    """The tensor/MUFU roofline of alu_roofline for a summed work record w."""
    t = ms / 1e3
    tens = (tensor_tflops or rates.get("bf16_tflops") or 1934.6) * 1e12
    t_ex2 = w["ex2"] / rates["ex2_per_s"]
    t_ten = (w["distance_flops"] + w["contraction_flops"]) / tens
    t_fma = w["fp32_slots"] / rates["fp32_fma_per_s"]
    if t_ex2 >= t_ten:
        pipe, work, r, unit = "mufu_ex2", w["ex2"], rates["ex2_per_s"], "Tex2/s"
    else:
        pipe, work, r, unit = "tensor", w["distance_flops"] + w["contraction_flops"], tens, \
            "TFLOP/s"
    t_b = max(t_ex2, t_ten)
    return {"bound": "alu" if pipe == "mufu_ex2" else "tensor", "pipe": pipe, "kernel": kernel,
            "achieved": work / t / 1e12, "peak": r / 1e12, "unit": unit, "frac": t_b / t,
            "frac_simt": max(t_fma, t_ex2) / t, "frac_evaluated": 2.0 * t_b / t,
            "avg_ms": ms, "algorithmic": w}


PEAK_SOURCE = ("kpcg_probe_rates on this GPU in this process (dependent chains of one "
               "instruction kind on every SM, CUDA events): of measured")
_RATES = {}


def probed_rates(kpcg):
    """Measured FP32 FMA, MUFU ex2 and FP64 FMA rates of this GPU, once per process."""
    if not _RATES:
        _RATES.update(kpcg.probe_rates())
    return dict(_RATES)


def df_issue_efficiency(n, d, c, ms, rates):
    """How fully the double-float kernel issues its own instructions: its
    instruction model (per distinct entry: 16 per dimension for the exact
    difference, TwoProduct and TwoSum, 33 for the table-driven exp2, 12 per
    column for each of the row and the mirrored column) over the FP32 rate."""
    ops = n * (n + 1) / 2.0 * (16 * d + 33 + 24 * c)
    return ops / (ms / 1e3) / rates["fp32_fma_per_s"]


def df_kernel_name(d):
    """The double-float product's kernel at dimension d (the tensor-core
    distances of kv_tcds_kernel, one evaluation per pair of points, up to
    d = 10; the FP32-pipe kernel above)."""
    return ("kv_tcds_kernel (double-float, tensor-core distances, symmetric)" if d <= 10 else
            "kv_df_sym_kernel (double-float)")


def df_issue_eff(n, d, c, ms, rates, symmetric=True):
    """Issue efficiency of whichever double-float kernel runs at d.  The
    tensor-core-distance kernels' model: 67 FP32-pipe instructions per
    evaluated entry (double-float sum of the five level accumulators and
    log2 s^2, Tang's exp2) + 11 per column (TwoProduct/TwoSum row sum); the
    symmetric kernel evaluates n^2/2 + 64 n entries and adds 14 per column
    for the mirrored column sum (its product and its share of the shuffle
    butterfly), the one-sided kernel evaluates n^2."""
    if d > 10:
        return df_issue_efficiency(n, d, c, ms, rates)
    if symmetric:
        instr = (n * float(n) / 2 + 64.0 * n) * (67 + 25 * c)
    else:
        instr = n * float(n) * (67 + 11 * c)
    return instr / (ms / 1e3) / rates["fp32_fma_per_s"]


def nystrom_roofline(n, m, c, ms, hbm_gbs):
    """The Nystrom apply streams K_XU (n x m FP32 pairs) twice and reads and
    writes the n x c block: HBM-bound."""
    b = 2 * 8.0 * n * m + 3 * 8.0 * n * c
    t = ms / 1e3
    return {"bound": "hbm", "kernel": "Nystrom apply", "achieved": b / t / 1e9, "peak": hbm_gbs,
            "unit": "GB/s", "frac": b / t / 1e9 / hbm_gbs, "avg_ms": ms, "bytes": b}


def sm_clock_probe():
    """Start an nvidia-smi sampler; returns (stop_fn -> dict)."""
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    dev = os.environ.get("LOCAL_RANK", "0")
    try:
        proc = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}",
                                 "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return lambda: {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    lines = []

    def reader():
        for ln in proc.stdout:
            lines.append(ln.strip())

    th = threading.Thread(target=reader, daemon=True)
    th.start()

    def stop():
        proc.terminate()
        try:
            proc.wait(timeout=5)
        except Exception:
            proc.kill()
        th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}

    return stop


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, device=None):
    """Whole-job step time under torchrun: the slowest rank's, on every rank
    (one process per GPU; without a process group it is the value itself)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_problem(rank, n=None):
    """The headline workload's instance solved by one rank: replicas only, each
    rank its own seeded system and inducing subset, no data exchanged."""
    p = synthetic.config2(seed=rank, n=n if n else N_FULL)
    idx = synthetic.inducing_subset(p.n, min(M_INDUCING, p.n), seed=1 + rank)
    return p, idx


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------------ oracle
def oracle_sample(n=N_FULL, state=None):
    """Time the FP64 CPU oracle, as it stands, on a bounded sample of the
    workload and scale it to one whole solve.  Sample: the oracle's Nystrom
    set-up (m = 1024) on the first n/2 rows (its cost is linear in the rows
    once K_XU is far larger than the caches), doubled; one full-size product
    K_y v; one preconditioner apply on the n/2-row set-up, doubled.  Whole
    solve = set-up + (iterations + 2) x (product + apply), with the iteration
    count of the oracle's own complete run at this n.  `state` (a dict) keeps
    the set-up and its time between calls, so repeated samples time only the
    product and the apply."""
    import oracle
    if state is None:
        state = {}
    p = synthetic.config2(seed=0, n=n)
    ell, s2 = oracle.split_theta(p.log_theta, p.d, p.ard)
    half = n // 2
    if "P" not in state:
        idx = synthetic.inducing_subset(half, M_INDUCING, seed=1)
        t0 = time.perf_counter()
        state["P"] = oracle.Nystrom(p.X[:half], ell, s2, p.noise, idx)
        state["setup_half_s"] = time.perf_counter() - t0
    setup = state["setup_half_s"] * n / half
    t0 = time.perf_counter()
    oracle.kyv(p.X, ell, s2, p.noise, p.y)
    t_kv = time.perf_counter() - t0
    t0 = time.perf_counter()
    state["P"].apply(p.y[:half])
    t_ap = time.perf_counter() - t0
    per_iter = t_kv + t_ap * n / half
    rec_path = os.path.join(ROOT, "tests", "golden", f"oracle_pcg_n{n}.json")
    n_iter, src = None, None
    if os.path.exists(rec_path):
        with open(rec_path) as f:
            rec = json.load(f)
        n_iter, src = int(rec["iterations"]), os.path.relpath(rec_path, ROOT)
    est = setup + per_iter * (n_iter + 2) if n_iter else None
    return {
        "value": est,
        "unit": "s",
        "cores": oracle.num_threads(),
        "kind": "oracle",
        "sample": (f"FP64 oracle: Nystrom set-up (m={M_INDUCING}) on the first {half} rows "
                   f"({state['setup_half_s']:.1f} s, doubled), one full-size K_y v "
                   f"({t_kv:.2f} s) and one apply on the half set-up ({t_ap:.3f} s, doubled) "
                   f"at n={n}; whole solve = set-up + ({n_iter} + 2) x (product + apply)"
                   + (f" (iteration count from {src})" if src else " (no recorded count)")),
        "setup_s": setup,
        "s_per_iteration": per_iter,
    }


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    vals = []
    base = None
    state = {}  # the set-up sample is timed once; every step times a product and an apply
    for s in range(args.warmup + args.steps):
        base = oracle_sample(state=state)
        if s >= args.warmup:
            vals.append(base["value"])
    v = statistics.mean(vals) if vals and None not in vals else None
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3 if v else None,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {k: base[k] for k in ("kind", "cores", "sample")} | {"value": v,
                                                                               "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------- GPU
BATCH_WORKLOAD = ("64 ARD-RBF problems, n~LogU[512,16384], d~U{2..16}, l_r~LogU(0.3,3)*sqrt(d), "
                  "s^2~LogU(0.5,2), noise~LogU(1e-4,1e-1), X~N(0,I); y plus 8 Rademacher probes "
                  "each; Nystrom m_p=min(m_max,max(64,n_p/m_div)); tol 1e-8 rel per column")


GRAD_WORKLOAD = ("ARD-RBF n=45730 d=9, standardized Gaussian X, l_r=exp(N(0,0.5^2))*sqrt(d), s=1, "
                 "noise=1e-3; y plus t=16 Rademacher probes solved as one block; Nystrom m=512 "
                 "built in-step; tol 1e-8 rel per column; gradient of log p for all 11 parameters")


def run_grad(args):
    """One step: Nystrom set-up plus the stochastic gradient of Eq. 2 (one
    17-column block solve and the fused derivative products)."""
    import torch
    import paper_1602_06693_gb300 as kpcg

    world, rank, local = dist_setup()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    p = synthetic.config3(seed=rank)
    idx = synthetic.inducing_subset(p.n, 512, seed=2 + rank)
    prec = kpcg.KPCG_TC_IR if args.precision == "auto" else mode_id(kpcg, args.precision)
    opt = kpcg.default_options(precision=prec, profile=1, inner_shift=0.25, inner_tol=0.2)
    X = torch.from_numpy(p.X).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    R = torch.from_numpy(synthetic.rademacher(p.n, 16, 77 + rank)).to(dev).t().contiguous().t()
    s = kpcg.Solver(X, p.log_theta, p.noise, ard=True, options=opt)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        s.set_theta(p.log_theta, p.noise)
        s.precond(kpcg.KPCG_PREC_NYSTROM, len(idx), idx)
        return s.grad(y, R, tol=TOL)

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)
    stop_clock = sm_clock_probe()
    times = []
    for _ in range(args.steps):
        flush.fill_(2.0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g, _, info = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
    clocks = stop_clock()
    t_step = statistics.mean(times)
    line = {
        "metric": "time per stochastic log-likelihood gradient (17-RHS block solve + dK/dtheta.V)",
        "value": t_step, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32+f64", "data": "synthetic",
        "config": {"workload": GRAD_WORKLOAD, "precision": args.precision,
                   "l2": "flushed between steps (256 MB write)"},
        "solve": {"iters_total": info.iters_total, "outer_steps": info.outer_steps,
                  "max_rel_res_fp64": info.max_rel_res, "kv_inner_ms": info.kv_inner_ms,
                  "kv_inner_calls": info.kv_inner_calls, "kv_outer_ms": info.kv_outer_ms,
                  "kv_outer_calls": info.kv_outer_calls, "precond_ms": info.precond_ms,
                  "precond_calls": info.precond_calls, "step_times_s": times},
        "grad": [float(v) for v in g],
        "clocks": clocks,
        "gpu_launches": int(info.launches),
    }
    if rank == 0:
        print(json.dumps(line))
    s.close()


WARM_WORKLOAD = ("ARD-RBF n=131072 d=10 X~N(0,I); Adam lr 0.05 on (log l_1..10, log s^2, "
                 "log noise) from l=1, s=1, noise=0.1; gradients with 4 fresh Rademacher probes; "
                 "Nystrom m=512; network 12-256-256-4 on the 4 latest solutions, trained on the "
                 "first n_train steps; each later step solved warm and cold at the same theta "
                 "to tol 1e-8")


def run_warm(args):
    """A shortened hyperparameter trajectory (one bench step = the whole run):
    per-solve iterations and device time, warm-started by the trained network
    against cold-started PCG at the same theta."""
    import torch
    import paper_1602_06693_gb300 as kpcg
    from paper_1602_06693_gb300.warmstart import Trajectory

    world, rank, local = dist_setup()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    n_steps, n_train = args.traj_steps, args.traj_train
    p = synthetic.config5(seed=rank)
    X = torch.from_numpy(p.X).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    opt = kpcg.default_options(precision=kpcg.KPCG_TC_IR, inner_shift=0.25,
                               inner_tol=args.inner_tol if args.inner_tol else 0.02)
    s = kpcg.Solver(X, p.log_theta, p.noise, ard=True, options=opt)
    pidx = synthetic.inducing_subset(p.n, 512, seed=3 + rank)
    probes = lambda k: torch.from_numpy(synthetic.rademacher(p.n, 4, 5000 + k)).to(dev)
    params = synthetic.mlp_init(11, p.d + 2, 256, 256, 4)
    # the cold solve at the same theta (the comparison) on every k-th warm step
    cmp_every = args.traj_compare_every
    tr = Trajectory(s, y, pidx, probes, basis="snapshots", q=4, lr=0.05, n_train=n_train,
                    mlp_params=params, epochs=2000, mlp_lr=1e-3, tol=TOL, compare=True,
                    compare_every=cmp_every)
    z0 = np.concatenate([p.log_theta, [math.log(p.noise)]])
    stop_clock = sm_clock_probe()
    t0 = time.perf_counter()
    recs = tr.run(z0, n_steps)
    wall = time.perf_counter() - t0
    clocks = stop_clock()
    warm_all = [r for r in recs if r.warm]
    if not warm_all:
        raise SystemExit("the trajectory has no warm-started step: it needs more steps than "
                         "--traj-train and more training steps than the 4 snapshots")
    # ratios over the steps that ran both solves at the same theta
    warm = [r for r in warm_all if r.cold_iters is not None]
    wi = [r.iters for r in warm]
    ci = [r.cold_iters for r in warm]
    wt = [r.solve_ms for r in warm]
    ct = [r.cold_ms for r in warm]
    line = {
        "metric": "per-solve time along the trajectory, learned warm start vs cold start",
        "value": statistics.mean(r.solve_ms for r in warm_all) / 1e3, "unit": "s", "n_gpus": 1,
        "steps": 1, "warmup": 0,
        "ms_per_step": wall * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32+f64 (network: fp32 train, bf16 infer)",
        "data": "synthetic",
        "config": {"workload": WARM_WORKLOAD, "trajectory_steps": n_steps, "n_train": n_train,
                   "cold_comparison_every": cmp_every,
                   "note": ("the specified trajectory" if (n_steps, n_train) == (200, 50) else
                            "shortened trajectory: the specified one has 200 steps, 50 for "
                            "training")},
        "warm": {"iters": wi, "solve_ms": wt, "mean_ms": statistics.mean(wt),
                 "all_steps_mean_ms": statistics.mean(r.solve_ms for r in warm_all),
                 "all_steps_iters": [r.iters for r in warm_all]},
        "training_steps": {"iters": [r.iters for r in recs if not r.warm],
                           "solve_ms": [r.solve_ms for r in recs if not r.warm]},
        "cold": {"iters": ci, "solve_ms": ct, "mean_ms": statistics.mean(ct)},
        "iteration_ratio": sum(wi) / max(1, sum(ci)),
        "time_ratio": sum(wt) / max(1e-9, sum(ct)),
        "max_rel_res": max(r.rel_res for r in recs),
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    s.close()


PREDICT_WORKLOAD = ("isotropic RBF n=4096 d=8 X~N(0,I), s=1, l=1, noise=1e-2, Nystrom m=256; "
                    "1024 test inputs X_*~N(0,I); predictive mean (FP64) and latent variance (one "
                    "double-float PCG solve with FP64 certification per block of 16 test points, "
                    "tol 1e-8)")


def run_predict(args):
    """One step: predictive mean and variance at 1024 test inputs."""
    import torch
    import paper_1602_06693_gb300 as kpcg

    world, rank, local = dist_setup()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    p = synthetic.config1(seed=rank)
    idx = synthetic.inducing_subset(p.n, 256, seed=1 + rank)
    Xs = torch.from_numpy(synthetic.rng(100 + rank).standard_normal((1024, p.d))
                          .astype(np.float32)).to(dev)
    s = kpcg.Solver(torch.from_numpy(p.X).to(dev), p.log_theta, p.noise, ard=False,
                    options=kpcg.default_options(precision=kpcg.KPCG_DF64))
    s.precond(kpcg.KPCG_PREC_NYSTROM, 256, idx)
    alpha, _, _, _ = s.solve(torch.from_numpy(p.y).to(dev), tol=TOL)
    for _ in range(args.warmup):
        s.predict(Xs, alpha, tol=TOL)
    torch.cuda.synchronize(dev)
    stop_clock = sm_clock_probe()
    times = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m, v, info = s.predict(Xs, alpha, tol=TOL)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
    clocks = stop_clock()
    line = {
        "metric": "time for predictive mean and variance at 1024 test inputs",
        "value": statistics.mean(times), "unit": "s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": {"workload": PREDICT_WORKLOAD},
        "solve": {"iters_total": info.iters_total, "max_rel_res_fp64": info.max_rel_res,
                  "step_times_s": times},
        "var_range": [float(v.min()), float(v.max())],
        "clocks": clocks, "gpu_launches": int(info.launches),
    }
    if rank == 0:
        print(json.dumps(line))
    s.close()


FIG1_LOG_ELL = (-1.0, -0.5, 0.0, 0.5, 1.0)
FIG1_LOG_NOISE = (-4.0, -3.0, -2.0, -1.0, 0.0)
FIG1_SHAPES = {"concrete": (1030, 8), "power": (9568, 4)}
FIG1_KINDS = ("none", "nystrom", "fitc", "pitc", "spectral", "block_jacobi")


def fig1_problem(shape, seed=0):
    """Synthetic stand-in of a dataset shape for the preconditioner comparison
    of Sec. 4: standardized Gaussian X, y = sum sin(x) + noise, isotropic kernel."""
    n, d = FIG1_SHAPES[shape]
    return synthetic.make_problem(n, d, seed, dist="standardized", ard=False, ell=1.0,
                                  name=f"{shape}-shaped n={n} d={d}")


def fig1_cell(kpcg, torch, dev, p, log_ell, log_noise, kind):
    """Iterations of (P)CG on one grid cell (Sec. 4): isotropic RBF with s^2 = 1,
    l = 10^log_ell, noise 10^log_noise, stop at ||r||^2 < n 1e-10, cap 100 000;
    Nystrom, FITC and PITC with m = sqrt(n) inducing points (PITC blocks of sqrt(n)
    rows), the random-feature preconditioner with m = sqrt(n) frequencies,
    block-Jacobi with blocks of sqrt(n)."""
    m = int(math.ceil(math.sqrt(p.n)))
    lt = np.array([log_ell * math.log(10.0), 0.0])
    opt = kpcg.default_options(precision=kpcg.KPCG_FP64, tol_mode=1, max_iter=100000)
    with kpcg.Solver(torch.from_numpy(p.X).to(dev), lt, 10.0 ** log_noise, ard=False,
                     options=opt) as s:
        if kind == "nystrom":
            s.precond(kpcg.KPCG_PREC_NYSTROM, m, synthetic.inducing_subset(p.n, m, seed=5))
        elif kind == "fitc":
            s.precond(kpcg.KPCG_PREC_FITC, m, synthetic.inducing_subset(p.n, m, seed=5))
        elif kind == "pitc":
            s.precond_pitc(m, synthetic.inducing_subset(p.n, m, seed=5), m)
        elif kind == "spectral":
            s.precond_spectral(synthetic.spectral_draws(m, p.d, seed=5))
        elif kind == "block_jacobi":
            s.precond(kpcg.KPCG_PREC_BLOCK_JACOBI, m)
        _, it, info, st = s.solve(torch.from_numpy(p.y).to(dev), tol=1e-10,
                                  raise_on_error=False)
    return int(it[0]), int(st)


def run_fig1(args):
    """The preconditioner comparison of Sec. 4 on synthetic data of the Concrete
    shape (and, with --fig1-power, the Power-plant shape): iteration counts over
    the (log10 l, log10 noise) grid and the gain log10(#PCG / #CG)."""
    import torch
    import paper_1602_06693_gb300 as kpcg

    world, rank, local = dist_setup()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    shapes = ["concrete"] + (["power"] if args.fig1_power else [])
    out = {}
    t0 = time.perf_counter()
    for shape in shapes:
        p = fig1_problem(shape)
        grid = []
        for le in FIG1_LOG_ELL:
            for ln in FIG1_LOG_NOISE:
                row = {"log10_ell": le, "log10_noise": ln}
                for kind in FIG1_KINDS:
                    it, st = fig1_cell(kpcg, torch, dev, p, le, ln, kind)
                    row[kind] = it
                    row[kind + "_status"] = st
                for kind in FIG1_KINDS[1:]:
                    row[kind + "_gain_log10"] = (math.log10(max(row[kind], 1) / max(row["none"], 1)))
                grid.append(row)
        out[shape] = grid
    wall = time.perf_counter() - t0
    line = {"metric": "PCG iterations over the (l, noise) grid, Sec. 4 comparison",
            "value": wall, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": wall * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "isotropic RBF, s^2=1, stop ||r||^2 < n 1e-10, cap 1e5; "
                                   "Nystrom, FITC, PITC m=sqrt(n) (PITC blocks sqrt(n)), random features m=sqrt(n), "
                                   "block-Jacobi b=sqrt(n); synthetic X of the dataset shapes",
                       "shapes": shapes},
            "grid": out}
    if rank == 0:
        print(json.dumps(line))


LAPLACE_M, LAPLACE_INNER_TOL = 128, 1e-4
LAPLACE_WORKLOAD = ("probit GP classification, EEG shape n=14979 d=14 (X~N(0,I) standardized, "
                    "y=sign(sum sin x) with 5% flipped), ARD l=sqrt(14), s^2=4; Laplace mode by "
                    "Newton from f=0 (stop |dPsi| <= 1e-12 |Psi|), each B = I + W^1/2 K W^1/2 "
                    "solve to 1e-10 from the previous step's z, preconditioned by the Nystrom "
                    "form of B (default m=128, rebuilt when W^1/2 drifts by >10%); default B-solve: "
                    "flexible CG around tensor-core inner PCG (inner_tol 1e-4); double-float K.V "
                    "for b, a, the outer directions and the certified residuals")


def laplace_oracle_sample(n_sample=2500):
    """The dense FP64 oracle on the first n_sample rows of the same workload
    (its cost is the O(n^3) Cholesky of B per Newton step), scaled to the full
    n by (n / n_sample)^3."""
    import oracle
    p = synthetic.eeg_shape(seed=0)
    ell, s2 = oracle.split_theta(p.log_theta, p.d, True)
    t0 = time.perf_counter()
    r = oracle.laplace_probit(p.X[:n_sample], ell, s2, p.y[:n_sample], tol=1e-12)
    t = time.perf_counter() - t0
    scale = (p.n / n_sample) ** 3
    return {"value": t * scale, "unit": "s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"dense FP64 oracle Newton on the first {n_sample} rows "
                       f"({r['steps']} steps, {t:.1f} s), scaled by (n/{n_sample})^3")}


def run_laplace(args):
    """One step: the Laplace mode of the EEG-shaped probit classifier."""
    import torch
    import paper_1602_06693_gb300 as kpcg

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    p = synthetic.eeg_shape(seed=rank)
    lm = args.laplace_m
    idx = synthetic.inducing_subset(p.n, lm, seed=12 + rank) if lm > 0 else None
    prec = kpcg.KPCG_TC_IR if args.precision == "auto" else mode_id(kpcg, args.precision)
    opt = kpcg.default_options(precision=prec)
    opt.inner_tol = args.inner_tol if args.inner_tol is not None else LAPLACE_INNER_TOL
    s = kpcg.Solver(torch.from_numpy(p.X).to(dev), p.log_theta, 1.0, ard=True, options=opt)
    if lm > 0:
        s.precond(kpcg.KPCG_PREC_NYSTROM, lm, idx)
    y = torch.from_numpy(p.y).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        s.laplace(y)
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)
    stop_clock = sm_clock_probe()
    times, info = [], None
    for _ in range(args.steps):
        flush.fill_(2.0)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f, a, info, st = s.laplace(y)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
    clocks = stop_clock()
    t_step = max_over_ranks(statistics.mean(times), dev)
    # the dominant kernel: the double-float K.V of one column (every CG
    # iteration of a B-solve and two per Newton step), timed alone
    v = torch.from_numpy(synthetic.rng(3).standard_normal(p.n)).to(dev)
    for _ in range(3):
        s.matvec_f64(v, impl=1)
    reps = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.matvec_f64(v, impl=1)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    kv_ms = e0.elapsed_time(e1) / reps
    rates = probed_rates(kpcg)
    roof = alu_roofline(df_kernel_name(p.d) + ", 1 column", p.n, p.d, 1, kv_ms, rates)
    roof.update({"traffic": None, "peak_source": PEAK_SOURCE,
                 "timing": f"{reps} back-to-back products, CUDA events on the launching stream",
                 "issue_efficiency": df_issue_eff(p.n, p.d, 1, kv_ms, rates)})
    # the inner product of the mixed B-solves: tensor-core K.V of one column
    roof_inner = None
    if prec == kpcg.KPCG_TC_IR:
        v32 = v.float()
        for _ in range(3):
            s.matvec_f32(v32, impl=1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            s.matvec_f32(v32, impl=1)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tc_ms = e0.elapsed_time(e1) / reps
        roof_inner = alu_roofline("kv_tc_kernel (tcgen05, 1 column)", p.n, p.d, 1, tc_ms, rates)
        roof_inner.update({"timing": roof["timing"], "peak_source": PEAK_SOURCE})
    # end to end: labels from pinned host memory, f back to the host
    yh = torch.from_numpy(p.y).pin_memory()
    fh = torch.empty(p.n, dtype=torch.float64).pin_memory()
    e2e_t = []
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(3.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        yd = yh.to(dev, non_blocking=True)
        fd, _, _, _ = s.laplace(yd, want_a=False)
        fh.copy_(fd, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_t.append(time.perf_counter() - t0)
    # predictions at 1024 test inputs from the mode (mean, variance, probability)
    pred = None
    if not args.no_predict:
        Xs = torch.from_numpy(synthetic.rng(200 + rank).standard_normal((1024, p.d))
                              .astype(np.float32)).to(dev)
        s.laplace_predict(y, f, a, Xs)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, pv, pp, pinfo = s.laplace_predict(y, f, a, Xs)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pred = {"test_points": 1024, "time_s": e0.elapsed_time(e1) / 1e3,
                "cg_iters_total": pinfo.cg_iters_total, "max_rel_res": pinfo.max_rel_res,
                "var_range": [float(pv.min()), float(pv.max())],
                "prob_range": [float(pp.min()), float(pp.max())]}
    extra = {}
    if rank == 0 and world == 1 and not args.skip_baselines:
        try:
            extra["cpu_baseline"] = laplace_oracle_sample()
        except Exception as e:
            extra["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    line = {
        "metric": "time to the Laplace mode of a probit GP classifier (EEG shape)",
        "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": LAPLACE_WORKLOAD, "m_b": lm, "inner_tol": opt.inner_tol,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "b_solves": ("double-float PCG" if prec in (kpcg.KPCG_DF64, kpcg.KPCG_FP64)
                                else "flexible CG around FP32/tensor-core inner PCG, "
                                     "double-float outer")},
        "laplace": {"status": st, "newton_steps": info.newton_steps,
                    "cg_iters_total": info.cg_iters_total, "psi": info.psi,
                    "precond_builds": info.precond_builds,
                    "max_rel_res": info.max_rel_res, "setup_ms": info.setup_ms,
                    "step_times_s": times,
                    "train_accuracy": float((torch.sign(f) == y).double().mean()),
                    "predict": pred},
        "roofline": roof, "roofline_inner": roof_inner, "clocks": clocks,
        "e2e": {"value": statistics.mean(e2e_t), "unit": "s",
                "h2d_bytes_per_step": int(yh.numel() * 8),
                "d2h_bytes_per_step": int(fh.numel() * 8)},
        "gpu_launches": int(info.launches),
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    s.close()


BATCH_SHIFT, BATCH_INNER_TOL = 0.25, 0.2


def run_batch(args):
    """64 independent uneven problems (9 right-hand sides each) in one batched
    mixed-precision solve; a step is one kpcg_batch_solve of the whole batch."""
    import torch
    import paper_1602_06693_gb300 as kpcg

    world, rank, local = dist_setup()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    problems = synthetic.config4_problems(seed=rank)
    probs, B = [], []
    c = 9
    for k, p in enumerate(problems):
        m = min(args.batch_m_max, max(64, p.n // args.batch_m_div))
        probs.append((torch.from_numpy(p.X).to(dev), p.log_theta, p.noise,
                      synthetic.inducing_subset(p.n, m, seed=300 + k)))
        B.append(np.column_stack([p.y, synthetic.rademacher(p.n, c - 1, 400 + k)]))
    opt = kpcg.default_options(precision=kpcg.KPCG_TC_IR, inner_shift=BATCH_SHIFT,
                               inner_tol=BATCH_INNER_TOL, max_iter=args.batch_max_iter,
                               max_outer=40, profile=1)
    if args.inner_shift is not None:
        opt.inner_shift = args.inner_shift
    if args.inner_tol is not None:
        opt.inner_tol = args.inner_tol
    b = kpcg.Batch(probs, options=opt)
    if args.probe != "none":
        b.set_tiling(8)
        Vf = b.empty(c, torch.float32)
        Vf.normal_()
        fn = b.matvec_f32 if args.probe == "kv" else b.precond_apply_f32
        fn(Vf, c)  # builds the preconditioners / operands
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ms = []
        for r in range(3):
            ev[0].record(stream)
            fn(Vf, c)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            ms.append(ev[0].elapsed_time(ev[1]))
        print(json.dumps({"probe": args.probe, "ms": ms, "workload": BATCH_WORKLOAD,
                          "m_max": args.batch_m_max, "m_div": args.batch_m_div}))
        b.close()
        return
    G, ctas, tune_ms = b.tune(c)
    Bb = b.block(B)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    # one profiled solve (kernel by kernel, CUDA events per kind) for the split;
    # the timed solves replay the inner iterations from captured CUDA graphs
    _, _, _, pinfo, _ = b.solve(Bb, c, tol=TOL, raise_on_error=False)
    opt.profile = 0
    b.set_options(opt)
    for _ in range(args.warmup):
        b.solve(Bb, c, tol=TOL, raise_on_error=False)
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)
    stop_clock = sm_clock_probe()
    times = []
    for _ in range(args.steps):
        flush.fill_(2.0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        X, iters, rel, info, st = b.solve(Bb, c, tol=TOL, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
    clocks = stop_clock()
    t_step = statistics.mean(times)
    # batched tensor-core product: per entry one ex2 and c FMAs on the FP32
    # side.  Inside the solve, converged problems are skipped, so the average
    # call does less than a full product; time one full product instead (all
    # problems, the tuned tiling; staging and reduction included).
    entries = float(sum(p.n ** 2 for p in problems))
    Vf = b.empty(c, torch.float32)
    Vf.normal_()
    for _ in range(2):
        b.matvec_f32(Vf, c)
    torch.cuda.synchronize(dev)
    ef0 = torch.cuda.Event(enable_timing=True)
    ef1 = torch.cuda.Event(enable_timing=True)
    ef0.record(stream)
    for _ in range(5):
        b.matvec_f32(Vf, c)
    ef1.record(stream)
    torch.cuda.synchronize(dev)
    avg_ms = ef0.elapsed_time(ef1) / 5
    ef0.record(stream)
    for _ in range(5):
        b.precond_apply_f32(Vf, c)
    ef1.record(stream)
    torch.cuda.synchronize(dev)
    precond_full_ms = ef0.elapsed_time(ef1) / 5
    rates = probed_rates(kpcg)
    rates["bf16_tflops"] = float(measured_peaks().get("bf16_tflops", 1934.6))
    works = [kv_algorithmic(q.n, q.d, c) for q in problems]
    wsum = {k: sum(w[k] for w in works) for k in works[0]}
    # end to end from pinned host buffers through the public API
    Bh = Bb.cpu().pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    Bd = Bh.to(dev, non_blocking=True)
    Xd, _, _, _, _ = b.solve(Bd, c, tol=TOL, raise_on_error=False)
    Xh.copy_(Xd, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    line = {
        "metric": "time to solve 64 uneven problems (9 RHS each) to rel-res 1e-8",
        "value": t_step, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32+f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "l2": "flushed between steps (256 MB write)",
                   "preconditioners": "built at the first solve (warm-up), reused",
                   "inner_shift": opt.inner_shift, "inner_tol": opt.inner_tol,
                   "m_max": args.batch_m_max, "m_div": args.batch_m_div,
                   "tiles_per_item": G, "ctas": ctas, "tune_ms": tune_ms},
        "solve": {"status": st, "iters_total": info.iters_total, "outer_steps": info.outer_steps,
                  "max_rel_res_fp64": float(rel.max()), "inner_iterations_in_graphs": True,
                  "precond_full_apply_ms": precond_full_ms, "kv_full_product_ms": avg_ms,
                  "step_times_s": times,
                  "profiled_solve": {"time_ms": pinfo.time_ms, "kv_inner_ms": pinfo.kv_inner_ms,
                                     "kv_inner_calls": pinfo.kv_inner_calls,
                                     "kv_outer_ms": pinfo.kv_outer_ms,
                                     "kv_outer_calls": pinfo.kv_outer_calls,
                                     "precond_ms": pinfo.precond_ms,
                                     "precond_calls": pinfo.precond_calls}},
        "roofline": roofline_from_work("kv_tc_batch_kernel (+stage, reduce), full product",
                                       wsum, avg_ms, rates)
        | {"traffic": None, "peak_source": PEAK_SOURCE, "evaluated_entries": entries},
        "clocks": clocks,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(Bh.numel() * 8),
                "d2h_bytes_per_step": int(Xh.numel() * 8)},
        "gpu_launches": int(info.launches),
    }
    if rank == 0:
        print(json.dumps(line))
    b.close()


def solve_options(kpcg, mode, **kw):
    o = dict(MODE_OPTS[mode])
    o.update(kw)
    return kpcg.default_options(precision=mode_id(kpcg, mode), **o)


def timed(stream, fn):
    """(result, ms) of fn() between two CUDA events on `stream`."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    e1.synchronize()
    return r, e0.elapsed_time(e1)


def solve_once(kpcg, X, y, p, idx, opt, stream, kind="nystrom", size=M_INDUCING, tol=TOL):
    """Build the preconditioner and solve from scratch; returns (info, status,
    set-up ms, total ms)."""
    s = kpcg.Solver(X, p.log_theta, p.noise, ard=True, options=opt)
    try:
        k = kpcg.KPCG_PREC_NYSTROM if kind == "nystrom" else kpcg.KPCG_PREC_BLOCK_JACOBI
        _, set_ms = timed(stream, lambda: s.precond(k, size, idx if kind == "nystrom" else None))
        (x, _, info, st), sol_ms = timed(stream, lambda: s.solve(y, tol=tol, raise_on_error=False))
        return info, st, set_ms, set_ms + sol_ms
    finally:
        s.close()


DTYPES = {"tc_ir": "bf16x3 exponent, f32 inner, f64 outer (double-float directions, fp64 "
                   "certified residual)",
          "fp32_ir": "f32 inner, f64 outer", "xf_ir": "f32 inner (exact differences), f64 outer",
          "tcx_ir": "sliced bf16 exponent, f32 inner, f64 outer",
          "df64": "double-float iterations, fp64 certified residual", "fp64": "f64"}
KV_NAMES = {"tc_ir": "kv_tcs_kernel (tcgen05 exponent, symmetric tile pairs)",
            "tcx_ir": "kv_tcx_kernel (tcgen05 sliced exponent, compensated contraction)",
            "fp32_ir": "kv_simt_kernel<float>", "xf_ir": "kv_xf_sym_kernel (exact differences)",
            "df64": df_kernel_name(D), "fp64": "kv_f64_sym_kernel (FP64)"}
# DRAM bytes per launch from ncu captures at n = 16384, by kernel
# name, as a function of n: each kernel reads only its inputs from DRAM (the
# n x n work stays on chip), so the traffic grows like n.  A kernel changed
# since its capture has no entry.
KNOWN_TRAFFIC = {
    "kv_df_sym_kernel": lambda n: 2291712.0 * n / 16384,
    "kv_tc_kernel": lambda n: 4284000.0 * n / 16384,
    "kv_tcds_kernel": lambda n: 21168128.0 * n / 16384,
}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at n = 16384, "
                  "scaled by n (inputs only)")


def known_traffic(kernel, n):
    f = KNOWN_TRAFFIC.get(kernel.split(" ")[0])
    return f(n) if f else None


def run_solve(args):
    import torch
    import paper_1602_06693_gb300 as kpcg

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    mode = HEADLINE_PREC if args.precision == "auto" else args.precision
    extra_opts = {}
    if args.inner_shift is not None:
        extra_opts["inner_shift"] = args.inner_shift
    if args.inner_tol is not None:
        extra_opts["inner_tol"] = args.inner_tol
    rates = probed_rates(kpcg)
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    rates["bf16_tflops"] = float(measured_peaks().get("bf16_tflops", 1934.6))

    # replicas: each rank solves its own seeded instance of the same workload
    p, idx = replica_problem(rank, args.n)
    X = torch.from_numpy(p.X).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    opt = solve_options(kpcg, mode, profile=0, **extra_opts)
    solver = kpcg.Solver(X, p.log_theta, p.noise, ard=True, options=opt)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    set_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def step():
        solver.set_theta(p.log_theta, p.noise)  # drop the preconditioner: rebuilt in-step
        set_ev[0].record(stream)
        solver.precond(kpcg.KPCG_PREC_NYSTROM, M_INDUCING, idx)
        set_ev[1].record(stream)
        return solver.solve(y, tol=TOL, raise_on_error=False)

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)

    stop_clock = sm_clock_probe()
    times, setups, infos = [], [], []
    for _ in range(args.steps):
        flush.fill_(2.0)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, it, info, st = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        times.append(e0.elapsed_time(e1) / 1e3)
        setups.append(set_ev[0].elapsed_time(set_ev[1]))
        infos.append((info, st))
    clocks = stop_clock()
    t_step = max_over_ranks(statistics.mean(times), dev)
    info, st = infos[-1]

    # The same step with the library's profiler on: CUDA events on the
    # handle's stream around every product and apply (kernel by kernel, no
    # graph replay), run right after the timed region on the same inputs.
    popt = solve_options(kpcg, mode, profile=1, **extra_opts)
    flush.fill_(3.0)
    pinfo, pst, pset_ms, ptot_ms = solve_once(kpcg, X, y, p, idx, popt, stream)
    cats = {}
    if pinfo.kv_inner_calls:
        ms = pinfo.kv_inner_ms / pinfo.kv_inner_calls
        cats["kv_inner"] = alu_roofline(KV_NAMES[mode], p.n, D, 1, ms, rates,
                                        fp64=(mode == "fp64"))
        cats["kv_inner"].update(calls=pinfo.kv_inner_calls, total_ms=pinfo.kv_inner_ms)
        if mode == "df64":
            cats["kv_inner"]["issue_efficiency"] = df_issue_eff(p.n, D, 1, ms, rates)
    if pinfo.kv_outer_calls:
        ms = pinfo.kv_outer_ms / pinfo.kv_outer_calls
        cats["kv_outer"] = alu_roofline(df_kernel_name(D) + " (outer directions)",
                                        p.n, D, 1, ms, rates)
        cats["kv_outer"].update(calls=pinfo.kv_outer_calls, total_ms=pinfo.kv_outer_ms,
                                issue_efficiency=df_issue_eff(p.n, D, 1, ms, rates))
    if pinfo.resid_calls:
        ms = pinfo.resid_ms / pinfo.resid_calls
        cats["resid"] = alu_roofline("kv_f64_sym_kernel (native FP64 certified residual)",
                                     p.n, D, 1, ms, rates, fp64=True)
        cats["resid"].update(calls=pinfo.resid_calls, total_ms=pinfo.resid_ms)
    if pinfo.precond_calls:
        ms = pinfo.precond_ms / pinfo.precond_calls
        cats["precond"] = nystrom_roofline(p.n, M_INDUCING, 1, ms, hbm)
        cats["precond"].update(calls=pinfo.precond_calls, total_ms=pinfo.precond_ms)
    dom = max(cats, key=lambda k: cats[k]["total_ms"]) if cats else None
    roof = dict(cats[dom]) if dom else {}
    if roof:
        roof["peak_source"] = (PEAK_SOURCE if roof["bound"] == "alu" else
                               "MEASURED_PEAKS.json hbm_gbs (of measured)")
        roof["timing"] = ("average launch of this class from CUDA events on the handle's stream "
                          "in a profiled run of the same step right after the timed region")
        roof["traffic"] = known_traffic(roof["kernel"], p.n)
        roof["traffic_source"] = TRAFFIC_SOURCE if roof["traffic"] else None

    # end to end through the C ABI from host buffers
    Xh = torch.from_numpy(p.X).pin_memory()
    yh = torch.from_numpy(p.y).pin_memory()
    xh = torch.empty(p.n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    e2e_times = []
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(3.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Xd = Xh.to(dev, non_blocking=True)
        yd = yh.to(dev, non_blocking=True)
        s2 = kpcg.Solver(Xd, p.log_theta, p.noise, ard=True, options=opt)
        s2.precond(kpcg.KPCG_PREC_NYSTROM, M_INDUCING, idx)
        xs, _, _, _ = s2.solve(yd, tol=TOL, raise_on_error=False)
        xh.copy_(xs, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_times.append(time.perf_counter() - t0)
        s2.close()
    e2e = {"value": statistics.mean(e2e_times), "unit": "s",
           "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 8 + idx.nbytes),
           "d2h_bytes_per_step": int(xh.numel() * 8)}

    extra = {}
    if rank == 0 and world == 1 and not args.skip_baselines:
        extra["comparisons"] = comparisons(kpcg, X, y, p, idx, stream, mode, extra_opts, args)
        try:
            extra["cpu_baseline"] = oracle_sample()
        except Exception as e:  # the baseline never blocks the GPU line
            extra["cpu_baseline"] = {"value": None, "error": str(e)[:200]}

    launches_per_step = int(info.launches)  # counted by the library inside the solve
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[mode], "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "solver": mode, "inner_shift": opt.inner_shift, "inner_tol": opt.inner_tol,
                   "path": "production (CUDA-graph replay of CG chunks, profiling off)"},
        "solve": {"status": st, "iters_total": info.iters_total, "outer_steps": info.outer_steps,
                  "max_rel_res_fp64": info.max_rel_res,
                  "setup_ms": statistics.mean(setups), "step_times_s": times,
                  "profiled": {"status": pst, "total_ms": ptot_ms, "setup_ms": pset_ms,
                               "kv_inner_ms": pinfo.kv_inner_ms,
                               "kv_inner_calls": pinfo.kv_inner_calls,
                               "kv_outer_ms": pinfo.kv_outer_ms,
                               "kv_outer_calls": pinfo.kv_outer_calls,
                               "resid_ms": pinfo.resid_ms, "resid_calls": pinfo.resid_calls,
                               "precond_ms": pinfo.precond_ms,
                               "precond_calls": pinfo.precond_calls}},
        "roofline": roof,
        "kernels": cats,
        "peaks": {"probe": rates, "hbm_gbs": hbm,
                  "bf16_tflops": measured_peaks().get("bf16_tflops")},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches_per_step,
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def comparisons(kpcg, X, y, p, idx, stream, mode, extra_opts, args):
    """The same-GPU comparisons of the measurement plan: plain FP32 PCG (its
    floor and time to 1e-6), the headline solver's time to 1e-6, the
    block-Jacobi arm (b = 512) and the double-float solver, each from scratch
    (preconditioner set-up included)."""
    out = {}
    # plain FP32 PCG, same Nystrom preconditioner, no restarts: one solve per
    # tolerance; the floor is the best FP64-recomputed residual any of them left
    fp32 = []
    for tol in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
        o32 = kpcg.default_options(precision=kpcg.KPCG_FP32, max_iter=args.fp32_max_iter,
                                   max_restarts=0)
        info, st, set_ms, tot_ms = solve_once(kpcg, X, y, p, idx, o32, stream, tol=tol)
        fp32.append({"tol": tol, "status": st, "iters": info.iters_total,
                     "rel_res_fp64": info.max_rel_res, "time_s": tot_ms / 1e3})
    floor = min(r["rel_res_fp64"] for r in fp32)
    t6 = [r["time_s"] for r in fp32 if r["tol"] == 1e-6 and r["rel_res_fp64"] <= 1e-6]
    out["fp32_pcg"] = {"floor_rel_res_fp64": floor, "time_to_1e-6_s": t6[0] if t6 else None,
                       "reached_1e-8": any(r["rel_res_fp64"] <= 1e-8 for r in fp32),
                       "runs": fp32,
                       "note": f"plain FP32 PCG, Nystrom m={M_INDUCING}, capped at "
                               f"{args.fp32_max_iter} iterations, no restarts"}
    o = solve_options(kpcg, mode, profile=0, **extra_opts)
    info, st, set_ms, tot_ms = solve_once(kpcg, X, y, p, idx, o, stream, tol=1e-6)
    out["kpcg_time_to_1e-6_s"] = tot_ms / 1e3
    out["kpcg_to_1e-6"] = {"status": st, "iters": info.iters_total,
                           "rel_res_fp64": info.max_rel_res}
    ob = solve_options(kpcg, mode, profile=0, max_iter=args.bj_max_iter, **extra_opts)
    info, st, set_ms, tot_ms = solve_once(kpcg, X, y, p, None, ob, stream, kind="block_jacobi",
                                          size=512)
    out["block_jacobi_512"] = {"status": st, "time_s": tot_ms / 1e3, "setup_ms": set_ms,
                               "iters": info.iters_total, "outer_steps": info.outer_steps,
                               "rel_res_fp64": info.max_rel_res,
                               "note": f"same solver, block-Jacobi blocks of 512, at most "
                                       f"{args.bj_max_iter} iterations"}
    # the other solvers of the library on the same system, from scratch
    others = {"df64": "double-float PCG, FP64-certified", "xf_ir": "exact-difference FP32 inner",
              "tcx_ir": "sliced tensor-core inner"}
    for m, what in others.items():
        if m == mode:
            continue
        od = solve_options(kpcg, m, profile=0)
        info, st, set_ms, tot_ms = solve_once(kpcg, X, y, p, idx, od, stream)
        out[m] = {"what": what, "status": st, "time_s": tot_ms / 1e3, "iters": info.iters_total,
                  "outer_steps": info.outer_steps, "rel_res_fp64": info.max_rel_res,
                  "inner_shift": od.inner_shift, "inner_tol": od.inner_tol}
    return out


KV_IMPLS = {"f64": ("f64", 0, "kv_f64_sym_kernel (native FP64)"),
            "df": ("f64", 1, "kv_tcds_kernel (double-float, tensor-core distances, symmetric)"),
            "df1": ("f64", 4, "kv_tcd_kernel (double-float, tensor-core distances, every entry)"),
            "dfs": ("f64", 3, "kv_df_sym_kernel (double-float)"),
            "f32": ("f32", 0, "kv_simt_kernel<float>"),
            "tc": ("f32", 1, "kv_tc_kernel (tcgen05, BF16x3 exponent)"),
            "xf": ("f32", 3, "kv_xf_sym_kernel (exact differences)"),
            "tcx": ("f32", 4, "kv_tcx_kernel (tcgen05, sliced per-point-exact exponent)"),
            "tcv": ("f32", 5, "kv_tcv_kernel (tcgen05 exponent and tcgen05 contraction)"),
            "tcs": ("f32", 6, "kv_tcs_kernel (tcgen05 exponent, symmetric tile pairs)")}


def run_kv(args):
    """One K.V kernel alone on the benchmark's input distribution at --n
    points and --kv-cols columns: --warmup untimed then --steps timed
    products with CUDA events on the launching stream (inputs larger than L2
    at n >= 16384); a small target for profilers too."""
    import torch
    import paper_1602_06693_gb300 as kpcg

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    p = synthetic.config2(seed=0, n=args.n)
    kind, impl, kname = KV_IMPLS[args.kv_impl]
    s = kpcg.Solver(torch.from_numpy(p.X).to(dev), p.log_theta, p.noise, ard=True)
    c = args.kv_cols
    V = torch.from_numpy(synthetic.rng(4).standard_normal((c, p.n))).to(dev).t()
    if kind == "f32":
        V = V.float()
    mv = (lambda: s.matvec_f64(V, impl=impl)) if kind == "f64" else \
        (lambda: s.matvec_f32(V, impl=impl))
    for _ in range(args.warmup):
        mv()
    torch.cuda.synchronize(dev)
    stop_clock = sm_clock_probe()
    _, ms = timed(stream, lambda: [mv() for _ in range(args.steps)])
    clocks = stop_clock()
    ms /= args.steps
    rates = probed_rates(kpcg)
    rates["bf16_tflops"] = float(measured_peaks().get("bf16_tflops", 1934.6))
    roof = alu_roofline(kname, p.n, p.d, c, ms, rates, fp64=(args.kv_impl == "f64"))
    roof.update({"peak_source": PEAK_SOURCE, "traffic": known_traffic(kname, p.n),
                 "timing": f"{args.steps} back-to-back products, CUDA events on the stream"})
    if args.kv_impl in ("df", "df1"):
        roof["issue_efficiency"] = df_issue_eff(p.n, p.d, c, ms, rates,
                                                symmetric=(args.kv_impl == "df"))
    elif args.kv_impl == "dfs":
        roof["issue_efficiency"] = df_issue_efficiency(p.n, p.d, c, ms, rates)
    print(json.dumps({"metric": f"time per K.V product ({args.kv_impl}, c={c})", "value": ms / 1e3,
                      "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                      "vs_baseline": None, "data": "synthetic",
                      "config": {"workload": f"K.V of the n={p.n} uniform-cube ARD system"},
                      "roofline": roof, "peaks": rates, "clocks": clocks}))
    s.close()


PRECISION_SWEEP = (("fp32_ir", 0.25, 0.1), ("fp32_ir", 1.0, 0.1), ("fp32_ir", 4.0, 0.1),
                   ("tc_ir", 0.25, 0.1), ("tc_ir", 1.0, 0.1), ("tc_ir", 2.0, 0.1),
                   ("tc_ir", 4.0, 0.1), ("xf_ir", 0.25, 0.3), ("tcx_ir", 0.1, 0.5),
                   ("tcx_ir", 0.25, 0.3))


def run_precision(args):
    """The record behind the choice of solver for the headline system: for
    each reduced-precision product, the norm of its error operator
    ||K_op - K||_2 (power iteration against the native-FP64 product) and its
    error on a smooth (constant) and a rough (Rademacher) unit vector, at
    n = 4096, 16384 and --n; then the flexible-CG solve of the n = --n system
    for each (mode, inner shift, inner tolerance) of the sweep, with the worst
    relative residual after every outer step (KPCG_TRACE lines on stderr)."""
    import torch
    import paper_1602_06693_gb300 as kpcg

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ops = {"fp32": ("f32", 0), "tc": ("f32", 1), "xf_ex2": ("f32", 2), "xf_poly": ("f32", 3),
           "tcx": ("f32", 4), "df": ("f64", 1)}
    sizes = sorted({4096, 16384, args.n})
    recs = []
    for n in sizes:
        p = synthetic.config2(seed=0, n=n)
        s = kpcg.Solver(torch.from_numpy(p.X).to(dev), p.log_theta, p.noise, ard=True)

        def apply(name, v):
            kind, impl = ops[name]
            return (s.matvec_f64(v, impl=impl) if kind == "f64" else
                    s.matvec_f32(v.float(), impl=impl).double())

        ones = torch.ones(n, dtype=torch.float64, device=dev) / math.sqrt(n)
        rad = torch.from_numpy(synthetic.rademacher(n, 1, seed=9)[:, 0].copy()).to(dev)
        rad /= math.sqrt(n)
        ref1, ref2 = s.matvec_f64(ones, impl=0), s.matvec_f64(rad, impl=0)
        g = torch.Generator().manual_seed(5)
        for name in ops:
            v = torch.randn(n, generator=g, dtype=torch.float64).to(dev)
            v /= v.norm()
            est = 0.0
            for _ in range(12):
                w = apply(name, v) - s.matvec_f64(v, impl=0)
                est = float(w.norm())
                v = w / est
            recs.append({"n": n, "op": name, "opnorm": est, "opnorm_over_noise": est / p.noise,
                         "err_smooth": float((apply(name, ones) - ref1).norm()),
                         "err_rough": float((apply(name, rad) - ref2).norm())})
        s.close()
    p = synthetic.config2(seed=0, n=args.n)
    idx = synthetic.inducing_subset(p.n, M_INDUCING, seed=1)
    X = torch.from_numpy(p.X).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    solves = []
    for mode, shift, itol in PRECISION_SWEEP:
        opt = kpcg.default_options(precision=mode_id(kpcg, mode), inner_shift=shift,
                                   inner_tol=itol, max_outer=40, inner_max_iter=300)
        sys.stderr.write(f"=== {mode} inner_shift={shift} inner_tol={itol}\n")
        sys.stderr.flush()
        info, st, set_ms, tot_ms = solve_once(kpcg, X, y, p, idx, opt,
                                              torch.cuda.current_stream(dev))
        solves.append({"mode": mode, "inner_shift": shift, "inner_tol": itol, "status": st,
                       "time_s": tot_ms / 1e3, "outer_steps": info.outer_steps,
                       "inner_iters": info.iters_total, "rel_res_fp64": info.max_rel_res})
    print(json.dumps({"metric": "operator error and mixed-precision convergence", "value": None,
                      "unit": None, "config": {"workload": WORKLOAD},
                      "operators": recs, "solves": solves}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kpcg", choices=["kpcg", "reference"])
    ap.add_argument("--precision", default="auto",
                    choices=["auto", "tc_ir", "fp32_ir", "xf_ir", "tcx_ir", "df64", "fp64"])
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--skip-baselines", action="store_true")
    ap.add_argument("--fp32-max-iter", type=int, default=3000)
    ap.add_argument("--bj-max-iter", type=int, default=6000,
                    help="block-Jacobi comparison: iteration cap")
    ap.add_argument("--kv-impl", default="tcx", choices=sorted(KV_IMPLS),
                    help="kv: the kernel timed")
    ap.add_argument("--kv-cols", type=int, default=1, help="kv: columns of V")
    ap.add_argument("--workload", default="solve65k",
                    choices=["solve65k", "batch64", "grad45k", "warm131k", "predict4k", "fig1",
                             "laplace15k", "kv", "precision"],
                    help="solve65k: the headline single solve; batch64: 64 uneven problems")
    ap.add_argument("--batch-max-iter", type=int, default=20000,
                    help="batch64: cap on inner iterations (short runs for profiling)")
    ap.add_argument("--inner-shift", type=float, default=None,
                    help="batch64: shift of the inner operator, in units of each noise")
    ap.add_argument("--inner-tol", type=float, default=None)
    ap.add_argument("--batch-m-max", type=int, default=1024,
                    help="batch64: inducing points m_p = min(m_max, max(64, n_p / m_div))")
    ap.add_argument("--batch-m-div", type=int, default=4)
    ap.add_argument("--fig1-power", action="store_true", help="fig1: add the Power-plant shape")
    ap.add_argument("--laplace-m", type=int, default=LAPLACE_M,
                    help="laplace15k: inducing points of the preconditioner of B (0: none)")
    ap.add_argument("--no-predict", action="store_true",
                    help="laplace15k: skip the predictions (a short target for profilers)")
    ap.add_argument("--traj-steps", type=int, default=200, help="warm131k: trajectory length")
    ap.add_argument("--traj-train", type=int, default=50, help="warm131k: training steps")
    ap.add_argument("--traj-compare-every", type=int, default=10,
                    help="warm131k: a cold solve at the same theta on every k-th warm step")
    ap.add_argument("--probe", default="none", choices=["none", "kv", "precond"],
                    help="batch64: only time full batched products (kv) or preconditioner "
                         "applies (precond) and exit; a small target for profilers")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "grad45k":
        return run_grad(args)
    if args.workload == "warm131k":
        return run_warm(args)
    if args.workload == "predict4k":
        return run_predict(args)
    if args.workload == "fig1":
        return run_fig1(args)
    if args.workload == "laplace15k":
        return run_laplace(args)
    if args.workload == "kv":
        return run_kv(args)
    if args.workload == "precision":
        return run_precision(args)
    return run_solve(args)


if __name__ == "__main__":
    main()
