#!/usr/bin/env python
"""Benchmark: PCG time-to-relative-residual 1e-8 on the n = 65536 kernel system.

Workload (one "step"): the ARD-RBF system (K + sigma^2 I) alpha = y with
n = 65536, d = 8, X ~ U[0,1]^8, l_r ~ LogUniform(0.3, 3), s = 1, sigma^2 = 1e-4
(seeded, synthetic), Nystrom preconditioner with m = 1024 random inducing
points built inside the step, solved to ||y - K_y alpha|| <= 1e-8 ||y|| by the
mixed-precision solver (outer flexible CG in FP64, inner FP32 PCG).  Inputs are
resident in HBM when the timed region starts; L2 is flushed between steps.

Printed: one JSON line with the time per solve (seconds, lower is better), the
end-to-end time through the C ABI from host buffers, the roofline of the
dominant kernel, the FP64 CPU oracle's time on a bounded sample of the same
workload, and the plain-FP32 PCG comparison on the same GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kpcg|reference]
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
# Algorithmic work of one double-float K.V, in FP32-pipe instructions.  K is
# symmetric, so each of the n(n+1)/2 distinct entries is evaluated once: per
# dimension 16 (exact difference, three-part low difference, TwoProduct, two
# FMAs, TwoSum into the exponent) plus 33 for the table-driven exp2 of a
# double-float; every (i, j) then costs 12 per right-hand side (split product
# and TwoSum accumulation).
def df_ops_per_product(n, d, c):
    return n * (n + 1) / 2 * (16 * d + 33) + float(n) * n * 12 * c


# Native-FP64 kernel: d subtractions and d FMAs for the distance, the FP64 exp
# (counted as one operation) and c FMAs.
def fp64_ops_per_entry(d, c):
    return 2 * d + 1 + c


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
def oracle_sample(n=N_FULL, iters=2):
    """Time the FP64 CPU oracle on a bounded sample of the workload: its Nystrom
    set-up plus `iters` PCG iterations at full size.  Scaled to a whole solve
    with the iteration count the oracle's own complete run recorded."""
    import oracle
    p = synthetic.config2(seed=0, n=n)
    ell, s2 = oracle.split_theta(p.log_theta, p.d, p.ard)
    idx = synthetic.inducing_subset(n, M_INDUCING, seed=1)
    t0 = time.perf_counter()
    P = oracle.Nystrom(p.X, ell, s2, p.noise, idx)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.pcg(p.X, ell, s2, p.noise, p.y, precond=P, tol=1e-30, max_iter=iters)
    t_iters = time.perf_counter() - t0
    # or_pcg also spends one K_y x for r0 and one for the final residual: iters + 2 products
    per_iter = t_iters / (iters + 2)
    rec_path = os.path.join(ROOT, "tests", "golden", f"oracle_pcg_n{n}.json")
    n_iter, src = None, None
    if os.path.exists(rec_path):
        with open(rec_path) as f:
            rec = json.load(f)
        n_iter, src = int(rec["iterations"]), os.path.relpath(rec_path, ROOT)
    est = t_setup + per_iter * (n_iter + 2) if n_iter else None
    return {
        "value": est,
        "unit": "s",
        "cores": oracle.num_threads(),
        "kind": "oracle",
        "sample": (f"FP64 oracle Nystrom set-up + {iters} PCG iterations at n={n} "
                   f"({t_setup:.1f} s + {t_iters:.1f} s); whole solve = set-up + "
                   f"{n_iter} iterations x {per_iter:.2f} s"
                   + (f" (iteration count from {src})" if src else " (no recorded count)")),
        "setup_s": t_setup,
        "s_per_iteration": per_iter,
    }


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    vals = []
    base = None
    for s in range(args.warmup + args.steps):
        base = oracle_sample(iters=1)
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
    prec = {"auto": kpcg.KPCG_TC_IR, "tc_ir": kpcg.KPCG_TC_IR, "df64": kpcg.KPCG_DF64,
            "fp32_ir": kpcg.KPCG_FP32_IR, "fp64": kpcg.KPCG_FP64}[args.precision]
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
    tr = Trajectory(s, y, pidx, probes, basis="snapshots", q=4, lr=0.05, n_train=n_train,
                    mlp_params=params, epochs=2000, mlp_lr=1e-3, tol=TOL, compare=True)
    z0 = np.concatenate([p.log_theta, [math.log(p.noise)]])
    stop_clock = sm_clock_probe()
    t0 = time.perf_counter()
    recs = tr.run(z0, n_steps)
    wall = time.perf_counter() - t0
    clocks = stop_clock()
    warm = [r for r in recs if r.warm]
    wi = [r.iters for r in warm]
    ci = [r.cold_iters for r in warm]
    wt = [r.solve_ms for r in warm]
    ct = [r.cold_ms for r in warm]
    line = {
        "metric": "per-solve time along the trajectory, learned warm start vs cold start",
        "value": statistics.mean(wt) / 1e3, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": wall * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32+f64 (network: fp32 train, bf16 infer)",
        "data": "synthetic",
        "config": {"workload": WARM_WORKLOAD, "trajectory_steps": n_steps, "n_train": n_train,
                   "note": "shortened trajectory: the specified one has 200 steps, 50 for training"},
        "warm": {"iters": wi, "solve_ms": wt, "mean_ms": statistics.mean(wt)},
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
    prec = {"auto": kpcg.KPCG_TC_IR, "df64": kpcg.KPCG_DF64, "fp32_ir": kpcg.KPCG_FP32_IR,
            "tc_ir": kpcg.KPCG_TC_IR, "fp64": kpcg.KPCG_FP64}[args.precision]
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
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    ops = df_ops_per_product(p.n, p.d, 1)
    peak = 152 * 128 * sm_max * 1e6 / 1e12
    roof = {"bound": "alu", "kernel": "kv_df_sym_kernel (double-float K.V, 1 column)",
            "achieved": ops / (kv_ms / 1e3) / 1e12, "peak": peak, "unit": "Top/s",
            "frac": ops / (kv_ms / 1e3) / 1e12 / peak, "traffic": None,
            "peak_source": (f"FP32 pipe issue rate: 152 SMs x 128 lanes x {sm_max:.0f} MHz "
                            "(unit counts and max clock)"),
            "avg_ms": kv_ms, "ops_per_call": ops,
            "timing": f"{reps} back-to-back products, CUDA events on the launching stream"}
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
        # the exponent comes from the tensor cores; each of the n^2 entries then
        # takes one ex2 on the special-function units (16 per SM per clock)
        tc_ops = float(p.n) * p.n
        mufu = 152 * 16 * sm_max * 1e6 / 1e12
        roof_inner = {"bound": "alu", "kernel": "kv_tc_kernel (tcgen05, 1 column)",
                      "achieved": tc_ops / (tc_ms / 1e3) / 1e12, "peak": mufu, "unit": "Tex2/s",
                      "frac": tc_ops / (tc_ms / 1e3) / 1e12 / mufu, "avg_ms": tc_ms,
                      "ops_per_call": tc_ops, "timing": roof["timing"],
                      "peak_source": (f"ex2 issue: 152 SMs x 16 per clock x {sm_max:.0f} MHz "
                                      "(unit counts and max clock)")}
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
    ops = entries * (c + 1)
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
    sm_max = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = 152 * 128 * sm_max * 1e6 / 1e12
    achieved = ops / (avg_ms / 1e3) / 1e12
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
        "roofline": {"bound": "alu", "kernel": "kv_tc_batch_kernel (+stage, reduce), full product",
                     "achieved": achieved, "peak": peak, "unit": "Top/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": f"FP32 pipe issue rate 152 x 128 x {sm_max:.0f} MHz (unit counts)",
                     "ops_per_call": ops, "avg_ms": avg_ms},
        "clocks": clocks,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(Bh.numel() * 8),
                "d2h_bytes_per_step": int(Xh.numel() * 8)},
        "gpu_launches": int(info.launches),
    }
    if rank == 0:
        print(json.dumps(line))
    b.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kpcg", choices=["kpcg", "reference"])
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--skip-baselines", action="store_true")
    ap.add_argument("--fp32-max-iter", type=int, default=3000)
    ap.add_argument("--workload", default="solve65k",
                    choices=["solve65k", "batch64", "grad45k", "warm131k", "predict4k", "fig1",
                             "laplace15k"],
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
    ap.add_argument("--traj-steps", type=int, default=24, help="warm131k: trajectory length")
    ap.add_argument("--traj-train", type=int, default=12, help="warm131k: training steps")
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

    import torch
    import paper_1602_06693_gb300 as kpcg

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    prec = {"auto": kpcg.KPCG_DF64, "df64": kpcg.KPCG_DF64, "fp32_ir": kpcg.KPCG_FP32_IR,
            "tc_ir": kpcg.KPCG_TC_IR, "fp64": kpcg.KPCG_FP64}[args.precision]

    # replicas: each rank solves its own seeded instance of the same workload
    p, idx = replica_problem(rank, args.n)
    X = torch.from_numpy(p.X).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    opt = kpcg.default_options(precision=prec, profile=1)
    solver = kpcg.Solver(X, p.log_theta, p.noise, ard=True, options=opt)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        solver.set_theta(p.log_theta, p.noise)  # drop the preconditioner: rebuilt in-step
        solver.precond(kpcg.KPCG_PREC_NYSTROM, M_INDUCING, idx)
        x, it, info, st = solver.solve(y, tol=TOL, raise_on_error=False)
        return x, it, info, st

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize(dev)

    stop_clock = sm_clock_probe()
    times, infos = [], []
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
        infos.append((info, st))
    clocks = stop_clock()
    t_step = max_over_ranks(statistics.mean(times), dev)
    info, st = infos[-1]

    # roofline of the dominant kernel class, from the library's event timers
    cats = {"kv_inner": (info.kv_inner_ms, info.kv_inner_calls),
            "kv_outer_fp64": (info.kv_outer_ms, info.kv_outer_calls),
            "precond_apply": (info.precond_ms, info.precond_calls)}
    dom = max(cats, key=lambda k: cats[k][0])
    ms, calls = cats[dom]
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    if dom.startswith("kv"):
        entries = float(p.n) ** 2
        if dom == "kv_inner" and prec == kpcg.KPCG_DF64:
            ops = df_ops_per_product(p.n, D, 1)
            peak = 152 * 128 * sm_max * 1e6 / 1e12
            peak_src = (f"FP32 pipe issue rate: 152 SMs x 128 lanes x {sm_max:.0f} MHz "
                        "(unit counts and max clock; no measured FP32 figure)")
            kname = "kv_df_sym_kernel (double-float K.V, symmetric tile pairs)"
        else:
            ops = fp64_ops_per_entry(D, 1) * entries
            peak = 1.25 / 2  # 1.25 TFLOP/s nominal FP64 = 0.625 T FMA-class op/s
            peak_src = "nominal GB300 FP64 rate, 1.25 TFLOP/s = 0.625 Top/s"
            kname = "kv_simt_kernel<double> (native FP64 K.V)"
        achieved = ops / (ms / calls / 1e3) / 1e12
        traffic, tsrc = None, None
        if dom == "kv_inner" and prec == kpcg.KPCG_DF64:
            # ncu capture at n = 16384 (profiles/kv_df_sym_kernel_n16384.md): 2.29 MB of
            # DRAM reads, 0 writes; the kernel re-reads nothing from DRAM, so its traffic
            # is its inputs and grows like n, not n^2
            traffic = 2.29e6 * p.n / 16384
            tsrc = "dram read+write per launch, ncu at n=16384 scaled by n (inputs only)"
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "Top/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_source": tsrc, "peak_source": peak_src, "calls": calls,
                "avg_ms": ms / calls, "ops_per_call": ops}
    else:
        # Nystrom apply streams K_XU (n x m FP32) twice and reads/writes n-vectors
        bytes_ = 2 * 4.0 * p.n * M_INDUCING + 3 * 8.0 * p.n
        achieved = bytes_ / (ms / calls / 1e3) / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"bound": "hbm", "kernel": "Nystrom apply", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "calls": calls,
                "avg_ms": ms / calls}

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
        # plain FP32 PCG on the same GPU, same preconditioner
        o32 = kpcg.default_options(precision=kpcg.KPCG_FP32, max_iter=args.fp32_max_iter,
                                   max_restarts=0)
        s32 = kpcg.Solver(X, p.log_theta, p.noise, ard=True, options=o32)
        t0 = time.perf_counter()
        s32.precond(kpcg.KPCG_PREC_NYSTROM, M_INDUCING, idx)
        x32, it32, inf32, st32 = s32.solve(y, tol=TOL, raise_on_error=False)
        torch.cuda.synchronize(dev)
        t32 = time.perf_counter() - t0
        extra["fp32_pcg"] = {"status": st32, "time_s": t32, "iters": int(inf32.iters_total),
                             "final_rel_res_fp64": inf32.max_rel_res,
                             "reached_tol": bool(st32 == 0),
                             "note": f"plain FP32 PCG, capped at {args.fp32_max_iter} iterations"}
        s32.close()
        try:
            extra["cpu_baseline"] = oracle_sample()
        except Exception as e:  # the baseline never blocks the GPU line
            extra["cpu_baseline"] = {"value": None, "error": str(e)[:200]}

    launches_per_step = int(info.launches)  # counted by the library inside the solve
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "precision": args.precision},
        "solve": {"status": st, "iters_total": info.iters_total, "outer_steps": info.outer_steps,
                  "max_rel_res_fp64": info.max_rel_res, "setup_ms": info.setup_ms,
                  "kv_inner_ms": info.kv_inner_ms, "kv_inner_calls": info.kv_inner_calls,
                  "kv_outer_ms": info.kv_outer_ms, "kv_outer_calls": info.kv_outer_calls,
                  "precond_ms": info.precond_ms, "precond_calls": info.precond_calls,
                  "step_times_s": times},
        "roofline": roof,
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


if __name__ == "__main__":
    main()
