"""Run the FP64 oracle's PCG (Algorithm 1, Nystrom preconditioner of Sec. 3.1)
to completion on the full n = 65536, d = 8, noise 1e-4 uniform-cube ARD
workload and record its iteration count, final residual and residual history.

Calls only ``oracle`` and ``synthetic``.  The benchmark's CPU baseline times a
bounded sample of the same oracle run (set-up plus a few iterations) and
scales it to a whole solve with the iteration count stored here.

    OMP_NUM_THREADS=<cores> python tests/golden/make_oracle_pcg_run.py [n]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthetic  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 65536
    m = 1024
    p = synthetic.config2(seed=0, n=n)
    ell, s2 = oracle.split_theta(p.log_theta, p.d, p.ard)
    idx = synthetic.inducing_subset(n, m, seed=1)
    t0 = time.time()
    P = oracle.Nystrom(p.X, ell, s2, p.noise, idx)
    t_setup = time.time() - t0
    t0 = time.time()
    x, it, rel, rc, hist = oracle.pcg(p.X, ell, s2, p.noise, p.y, precond=P, tol=1e-8,
                                      max_iter=20000, history=True)
    t_solve = time.time() - t0
    out = {
        "workload": f"ard-rbf n={n} d=8 noise=1e-4 uniform-cube, seed 0; Nystrom m={m} seed 1",
        "tol": 1e-8,
        "iterations": int(it[0]),
        "status": rc,
        "final_rel_res": float(rel[0]),
        "setup_s": t_setup,
        "solve_s": t_solve,
        "threads": oracle.num_threads(),
        "history_every_10": [float(v) for v in hist[::10]],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_pcg_n{n}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "history_every_10"}))


if __name__ == "__main__":
    main()
