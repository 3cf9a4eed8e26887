"""Seeded synthetic inputs for the Gaussian-process systems the paper solves.

This module only draws random numbers (NumPy ``PCG64``) and lays them out: it
holds none of the method's arithmetic (no kernel entries, no solves).  Both
the FP64 CPU oracle and the CUDA path take their inputs from here, so a
parity test feeds the two sides byte-identical data.

Shapes and distributions follow the paper's workloads (Sec. 4 and Sec. 5:
UCI-sized problems, an RBF/ARD kernel, Eq. 1) as restated for the
benchmark suite; the UCI datasets themselves are not available, so every
workload is a synthetic stand-in of the same size and dimension.

Conventions
-----------
* ``X`` is float32, row-major ``n x d``.  Both sides read these exact float32
  values (the oracle widens them to float64).
* ``log_theta`` is float64: ``[log l_1, ..., log l_d, log s^2]`` for ARD, or
  ``[log l, log s^2]`` for the isotropic kernel.  ``noise`` is sigma^2 (the
  paper's lambda).
* Right-hand sides and probes are float64 column-major ``n x c`` arrays
  (``order='F'``).
* Rademacher probes take the values +-1 with probability 1/2 (Sec. 2.1).
* Inducing points are a sorted random subset of row indices drawn without
  replacement (Sec. 3.1; Sec. 5 draws them at random from the inputs).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "GPProblem",
    "rng",
    "make_problem",
    "config1",
    "config2",
    "config3",
    "config4_problems",
    "config5",
    "rademacher",
    "inducing_subset",
    "mlp_init",
    "spectral_draws",
    "classification_problem",
    "eeg_shape",
    "credit_shape",
]


def rng(seed: int) -> np.random.Generator:
    """The one generator used everywhere: NumPy PCG64 seeded by ``seed``."""
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclasses.dataclass
class GPProblem:
    """One kernel system ``(K(X,X|theta) + noise*I) alpha = y``."""

    X: np.ndarray  # float32 (n, d), C-contiguous
    y: np.ndarray  # float64 (n,)
    log_theta: np.ndarray  # float64 (d+1,) for ARD, (2,) for isotropic
    noise: float  # sigma^2 (paper's lambda)
    ard: bool
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    def lengthscales(self) -> np.ndarray:
        """Per-dimension lengthscales l_r (isotropic: one value repeated)."""
        ls = np.exp(self.log_theta[:-1])
        return ls if self.ard else np.full(self.d, ls[0])

    @property
    def s2(self) -> float:
        return float(math.exp(self.log_theta[-1]))


def _targets(g: np.random.Generator, X: np.ndarray, noise_sd: float = 0.1) -> np.ndarray:
    """y = sum_j sin(x_j) + N(0, noise_sd^2): a smooth signal plus white noise."""
    Xd = X.astype(np.float64)
    return np.sin(Xd).sum(axis=1) + noise_sd * g.standard_normal(X.shape[0])


def make_problem(n: int, d: int, seed: int, *, dist: str = "normal", ard: bool = True,
                 ell=None, s2: float = 1.0, noise: float = 1e-2, name: str = "") -> GPProblem:
    """A generic seeded problem; ``ell`` is a scalar, an array, or 'loguniform'."""
    g = rng(seed)
    if dist == "normal":
        X = g.standard_normal((n, d))
    elif dist == "uniform":
        X = g.random((n, d))
    elif dist == "standardized":
        X = g.standard_normal((n, d))
        X = (X - X.mean(axis=0)) / X.std(axis=0)
    else:
        raise ValueError(dist)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = _targets(g, X)
    if ell is None:
        ell = 1.0
    if isinstance(ell, str) and ell == "loguniform":
        ls = np.exp(g.uniform(math.log(0.3), math.log(3.0), size=d))
    else:
        ls = np.broadcast_to(np.asarray(ell, dtype=np.float64), (d,)).copy()
    if ard:
        log_theta = np.concatenate([np.log(ls), [math.log(s2)]])
    else:
        log_theta = np.array([math.log(ls[0]), math.log(s2)])
    return GPProblem(X=X, y=y, log_theta=log_theta.astype(np.float64), noise=float(noise), ard=ard,
                     name=name)


def config1(seed: int = 0, n: int = 4096) -> GPProblem:
    """Isotropic RBF, s=1, l=1, sigma^2=1e-2, X ~ N(0, I_8), n=4096."""
    return make_problem(n, 8, seed, dist="normal", ard=False, ell=1.0, s2=1.0, noise=1e-2,
                        name=f"iso-rbf n={n} d=8 noise=1e-2")


def config2(seed: int = 0, n: int = 65536) -> GPProblem:
    """ARD RBF, l_r ~ LogUniform(0.3, 3), X ~ U[0,1]^8, sigma^2=1e-4, n=65536."""
    return make_problem(n, 8, seed, dist="uniform", ard=True, ell="loguniform", s2=1.0,
                        noise=1e-4, name=f"ard-rbf n={n} d=8 noise=1e-4")


def config3(seed: int = 0, n: int = 45730) -> GPProblem:
    """ARD RBF on standardized Gaussian X (n=45730, d=9), sigma^2=1e-3.

    Lengthscales l_r = exp(N(0, 0.5^2)) * sqrt(d), drawn after X and y.
    """
    g = rng(seed)
    d = 9
    X = g.standard_normal((n, d))
    X = (X - X.mean(axis=0)) / X.std(axis=0)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = _targets(g, X)
    ls = np.exp(0.5 * g.standard_normal(d)) * math.sqrt(d)
    log_theta = np.concatenate([np.log(ls), [0.0]])
    return GPProblem(X=X, y=y, log_theta=log_theta, noise=1e-3, ard=True,
                     name=f"ard-rbf n={n} d=9 noise=1e-3")


def config4_problems(seed: int = 0, count: int = 64, n_lo: int = 512, n_hi: int = 16384):
    """Independent uneven problems: n ~ LogUniform[n_lo, n_hi], d ~ U{2..16}.

    l_r ~ LogUniform(0.3, 3) * sqrt(d), s^2 ~ LogUniform(0.5, 2),
    sigma^2 ~ LogUniform(1e-4, 1e-1), X ~ N(0, I_d).
    """
    g = rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(g.integers(2, 17))
        sub_seed = int(g.integers(0, 2**62))
        gk = rng(sub_seed)
        X = np.ascontiguousarray(gk.standard_normal((n, d)), dtype=np.float32)
        y = _targets(gk, X)
        ls = np.exp(gk.uniform(math.log(0.3), math.log(3.0), size=d)) * math.sqrt(d)
        s2 = math.exp(gk.uniform(math.log(0.5), math.log(2.0)))
        noise = math.exp(gk.uniform(math.log(1e-4), math.log(1e-1)))
        log_theta = np.concatenate([np.log(ls), [math.log(s2)]])
        out.append(GPProblem(X=X, y=y, log_theta=log_theta, noise=noise, ard=True,
                             name=f"batch[{k}] n={n} d={d}"))
    return out


def config5(seed: int = 0, n: int = 131072) -> GPProblem:
    """n=131072, d=10, X ~ N(0, I); start of the trajectory: l=1, s=1, sigma^2=0.1."""
    return make_problem(n, 10, seed, dist="normal", ard=True, ell=1.0, s2=1.0, noise=0.1,
                        name=f"ard-rbf n={n} d=10 trajectory")


def rademacher(n: int, t: int, seed: int) -> np.ndarray:
    """n x t probe matrix of +-1 (float64, column-major), P(+1) = P(-1) = 1/2."""
    g = rng(seed)
    bits = g.integers(0, 2, size=(t, n), dtype=np.int8)
    R = (2.0 * bits.astype(np.float64) - 1.0).T
    return np.asfortranarray(R)


def inducing_subset(n: int, m: int, seed: int) -> np.ndarray:
    """Sorted int64 indices of m distinct rows out of n."""
    if m > n:
        raise ValueError("m > n")
    g = rng(seed)
    return np.sort(g.choice(n, size=m, replace=False)).astype(np.int64)


def mlp_init(seed: int, n_in: int, h1: int, h2: int, n_out: int) -> dict:
    """Xavier-uniform initial weights (zero biases), float64, for the
    warm-start network: W1 (h1, n_in), b1, W2 (h2, h1), b2, W3 (n_out, h2), b3."""
    g = rng(seed)

    def xavier(o, i):
        a = math.sqrt(6.0 / (i + o))
        return g.uniform(-a, a, size=(o, i))

    return {"W1": xavier(h1, n_in), "b1": np.zeros(h1), "W2": xavier(h2, h1),
            "b2": np.zeros(h2), "W3": xavier(n_out, h2), "b3": np.zeros(n_out)}


def spectral_draws(m: int, d: int, seed: int) -> np.ndarray:
    """m x d standard-normal draws (float64, row-major): the random part of the
    spectral points of the random-feature preconditioner (Sec. 3.2), which both
    sides scale by 1 / (2 pi l) themselves."""
    return np.ascontiguousarray(rng(seed).standard_normal((m, d)))


def classification_problem(n: int, d: int, seed: int, *, ell=None, s2: float = 4.0,
                           flip: float = 0.05, name: str = "") -> GPProblem:
    """Binary labels y = +-1 for probit GP classification (Sec. 2.2, App. B):
    X ~ N(0, I_d) standardized per column, y = sign(sum_j sin(x_j)), each label
    flipped with probability ``flip``; ``noise`` is unused by the classifier
    (set to 1).  ``ell`` defaults to sqrt(d), ARD."""
    g = rng(seed)
    X = g.standard_normal((n, d))
    X = (X - X.mean(axis=0)) / X.std(axis=0)
    X = np.ascontiguousarray(X, dtype=np.float32)
    s = np.sin(X.astype(np.float64)).sum(axis=1)
    y = np.where(s >= 0.0, 1.0, -1.0)
    y = np.where(g.random(n) < flip, -y, y)
    ls = np.full(d, math.sqrt(d)) if ell is None else \
        np.broadcast_to(np.asarray(ell, dtype=np.float64), (d,)).copy()
    log_theta = np.concatenate([np.log(ls), [math.log(s2)]])
    return GPProblem(X=X, y=y, log_theta=log_theta.astype(np.float64), noise=1.0, ard=True,
                     name=name)


def eeg_shape(seed: int = 0) -> GPProblem:
    """Stand-in of the EEG classification set's shape (n=14979, d=14, Sec. 5)."""
    return classification_problem(14979, 14, seed, name="probit n=14979 d=14 (EEG shape)")


def credit_shape(seed: int = 0) -> GPProblem:
    """Stand-in of the Credit classification set's shape (n=1000, d=24, App. C)."""
    return classification_problem(1000, 24, seed, name="probit n=1000 d=24 (Credit shape)")
