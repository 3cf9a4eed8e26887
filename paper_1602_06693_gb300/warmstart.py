"""Learned warm start of PCG along a hyperparameter trajectory.

Stochastic-gradient ascent on log p(y|theta) (gradient of Eq. 2 with the
Rademacher trace estimate of Sec. 2.1; the paper's optimiser is ADAGRAD with
N_r = 4 probes, Sec. 5, this driver uses Adam) visits theta_1, theta_2, ...,
and every step solves K_y(theta_k) alpha_k = y.  Algorithm 1 starts from an
initial iterate x0.  A small network maps the step's log-hyperparameters to
coefficients c on a basis B and PCG starts from x0 = B c; it still runs to the
same tolerance, so the network only moves the starting point.

Bases (kpcg_warm_*):
  * ``"snapshots"`` (default): the q most recent solutions of the trajectory,
    newest first.  Along the trajectory alpha(theta) moves smoothly, so a
    combination of recent solutions is close to the next one; the training
    target of step k is the least-squares combination of the q solutions
    before it.
  * ``"kernel"``: K(X, Z | theta) on m fixed inducing points; target = the
    least-squares fit of alpha_k.  alpha = K_y^{-1} y is dominated by its rough
    component, which a smooth kernel basis does not represent, so this basis
    saves few iterations even with exact coefficients; kept for comparison.

For the first ``n_train`` steps the driver records (theta_k, c*_k), then
trains the network (kpcg_mlp_train, FP32 Adam) and from then on predicts c in
BF16 (kpcg_mlp_forward).  The optimiser's few scalars (d + 2 log-parameters)
and the affine standardisation of the network's inputs and outputs are host
arithmetic; solves, gradients, fits, expansions and the network run in the
library.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import binding as _b


@dataclasses.dataclass
class StepRecord:
    step: int
    warm: bool
    iters: int        # PCG iterations of the alpha solve
    solve_ms: float   # device time of the alpha solve (CUDA events)
    rel_res: float
    log_theta: np.ndarray
    log_noise: float
    cold_iters: int | None = None  # a cold-started solve at the same theta (compare=True)
    cold_ms: float | None = None


class Trajectory:
    def __init__(self, solver: "_b.Solver", y, precond_idx, probes_fn, *, basis="snapshots",
                 q=4, basis_idx=None, lr=0.05, n_train=50, mlp_params=None, epochs=2000,
                 mlp_lr=1e-3, tol=1e-8, ridge=None, compare=False, compare_every=1):
        import torch

        self.torch = torch
        self.s = solver
        self.y = y
        self.precond_idx = np.asarray(precond_idx, dtype=np.int64)
        self.probes_fn = probes_fn
        self.lr = lr
        self.n_train = n_train
        self.epochs = epochs
        self.mlp_lr = mlp_lr
        self.tol = tol
        self.compare = compare
        self.compare_every = max(1, int(compare_every))
        self.basis = basis
        self.q = q
        if basis == "snapshots":
            self.s.warm_snapshots(q, 1e-10 if ridge is None else ridge)
        elif basis == "kernel":
            self.s.warm_basis(basis_idx, 1e-6 if ridge is None else ridge)
        else:
            raise ValueError(basis)
        self.n_seen = 0
        self.mlp_params = mlp_params
        self.mlp = None
        self.inputs, self.targets = [], []
        self.m1 = self.m2 = None
        self.t = 0
        self.records: list[StepRecord] = []

    # -- host-side standardisation of the network's inputs and outputs
    def _fit_scalers(self):
        Z = np.array(self.inputs)
        C = np.array(self.targets)
        self.z_mu, self.z_sd = Z.mean(0), np.maximum(Z.std(0), 1e-3)
        self.c_mu, self.c_sd = C.mean(0), np.maximum(C.std(0), 1e-12 + 1e-6 * np.abs(C).max())

    def train(self):
        torch = self.torch
        self._fit_scalers()
        Zs = (np.array(self.inputs) - self.z_mu) / self.z_sd
        Cs = (np.array(self.targets) - self.c_mu) / self.c_sd
        self.Xt = torch.from_numpy(Zs.astype(np.float32)).cuda()
        self.Tt = torch.from_numpy(Cs.astype(np.float32)).cuda()
        self.mlp = _b.MLP(self.mlp_params, max_batch=max(256, len(self.inputs)))
        return self.mlp.train(self.Xt, self.Tt, self.epochs, self.mlp_lr)

    def predict_x0(self, z):
        torch = self.torch
        zi = torch.from_numpy(((z - self.z_mu) / self.z_sd).astype(np.float32)[None, :]).cuda()
        cs = self.mlp.forward(zi, bf16=True)[0].double().cpu().numpy()
        c = torch.from_numpy(cs * self.c_sd + self.c_mu).cuda()
        return self.s.warm_expand(c)

    def _timed_solve(self, x0):
        torch = self.torch
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        alpha, it, info, _ = self.s.solve(self.y, tol=self.tol, X0=x0, raise_on_error=False)
        e1.record(st)
        torch.cuda.synchronize()
        return alpha, int(it[0]), e0.elapsed_time(e1), info.max_rel_res

    def step(self, k, z):
        """One trajectory step at z = [log_theta..., log noise]; returns the gradient."""
        s = self.s
        s.set_theta(z[:-1], math.exp(z[-1]))
        s.precond(_b.KPCG_PREC_NYSTROM, len(self.precond_idx), self.precond_idx)
        warm = self.mlp is not None
        cold_it = cold_ms = None
        if warm and self.compare and (k - self.n_train) % self.compare_every == 0:
            _, cold_it, cold_ms, _ = self._timed_solve(None)
        x0 = self.predict_x0(z) if warm else None
        alpha, it, ms, rel = self._timed_solve(x0)
        self.records.append(StepRecord(k, warm, it, ms, rel, np.array(z[:-1]), float(z[-1]),
                                       cold_it, cold_ms))
        if k < self.n_train and (self.basis == "kernel" or self.n_seen >= self.q):
            self.inputs.append(np.array(z))
            self.targets.append(s.warm_fit(alpha).cpu().numpy())
        if self.basis == "snapshots":
            s.warm_push(alpha)
        self.n_seen += 1
        g, _, _ = s.grad(self.y, self.probes_fn(k), tol=self.tol, alpha0=alpha)
        return g

    def run(self, z0, steps):
        z = np.array(z0, dtype=np.float64)
        self.m1 = np.zeros_like(z)
        self.m2 = np.zeros_like(z)
        for k in range(steps):
            if (k == self.n_train and self.mlp is None and self.mlp_params is not None
                    and self.inputs):
                self.train()
            g = self.step(k, z)
            # Adam ascent on log p
            self.t += 1
            self.m1 = 0.9 * self.m1 + 0.1 * g
            self.m2 = 0.999 * self.m2 + 0.001 * g * g
            mh = self.m1 / (1 - 0.9 ** self.t)
            vh = self.m2 / (1 - 0.999 ** self.t)
            z = z + self.lr * mh / (np.sqrt(vh) + 1e-8)
        return self.records
