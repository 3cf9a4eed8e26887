"""FP64 CPU oracle for preconditioned CG on kernel matrices.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline import this package; the library itself never does.  It shares no
code with the CUDA path.  The heavy loops live in ``kpcg_oracle.c`` (plain C,
FP64, OpenMP over rows); this module loads it with ctypes and assembles the
gradient of the log marginal likelihood (Eq. 2 with the stochastic trace of
Sec. 2.1) from its products.

It also restates, densely in NumPy for small n, the FITC, PITC and random-feature
preconditioners (Sec. 3.1, 3.2), the predictive mean and variance (Sec. 2.1), and the
probit Laplace approximation with its predictions (Sec. 2.2, Appendix B).

Every function cites the passage of the paper it restates.  Parameters are
taken in log space: ``log_theta = [log l_1..log l_d, log s^2]`` (ARD) or
``[log l, log s^2]`` (isotropic), noise sigma^2 separate.  Gradients are
d log p / d(log l_r), d/d(log s^2), d/d(log sigma^2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kpcg_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile ``kpcg_oracle.c`` into ``_liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_num_threads.restype = _int
            lib.or_gram.argtypes = [_d, _i64, _d, _i64, _int, _d, ctypes.c_double, _d]
            lib.or_kyv.argtypes = [_d, _i64, _int, _d, ctypes.c_double, ctypes.c_double,
                                   _d, _i64, _int, _d, _i64]
            lib.or_dkv.argtypes = [_d, _i64, _int, _d, ctypes.c_double, _d, _i64, _int, _d]
            lib.or_chol.argtypes = [_d, _i64]
            lib.or_chol.restype = _int
            lib.or_chol_solve.argtypes = [_d, _i64, _d, _i64, _int]
            lib.or_nys_setup.argtypes = [_d, _i64, _int, _d, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int64), _i64, _d, _d, _d]
            lib.or_nys_setup.restype = _int
            lib.or_nys_apply.argtypes = [_i64, _i64, ctypes.c_double, _d, _d, _d, _i64, _int,
                                         _d, _i64]
            lib.or_bj_setup.argtypes = [_d, _i64, _int, _d, ctypes.c_double, ctypes.c_double,
                                        _i64, _d]
            lib.or_bj_setup.restype = _int
            lib.or_bj_apply.argtypes = [_i64, _i64, _d, _d, _i64, _int, _d, _i64]
            lib.or_pcg.argtypes = [_d, _i64, _int, _d, ctypes.c_double, ctypes.c_double, _int,
                                   _d, _d, _i64, _d, _i64, _d, _i64, _int, ctypes.c_double, _int,
                                   _int, _d, _d, _i64, ctypes.POINTER(ctypes.c_int), _d, _d]
            lib.or_pcg.restype = _int
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(_d)


def _f64c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _f64f(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return np.asfortranarray(a)


def split_theta(log_theta, d: int, ard: bool):
    """(lengthscales[d], s2) from log parameters (Eq. 1)."""
    lt = np.asarray(log_theta, dtype=np.float64)
    ell = np.exp(lt[:-1]) if ard else np.full(d, np.exp(lt[0]))
    if ard and ell.shape[0] != d:
        raise ValueError("ARD log_theta needs d lengthscales")
    return np.ascontiguousarray(ell), float(np.exp(lt[-1]))


# ---------------------------------------------------------------------------
# Kernel entries and products (Eq. 1; Sec. 2.1)
# ---------------------------------------------------------------------------
def gram(X, Z, ell, s2) -> np.ndarray:
    """K(X, Z) with entries s2 * exp(-1/2 sum_r (x_r - z_r)^2 / l_r^2)  (Eq. 1)."""
    X = _f64c(X)
    Z = _f64c(Z)
    n, d = X.shape
    m = Z.shape[0]
    G = np.empty((n, m), dtype=np.float64)
    _load().or_gram(_p(X), n, _p(Z), m, d, _p(_f64c(ell)), float(s2), _p(G))
    return G


def kyv(X, ell, s2, noise, V) -> np.ndarray:
    """(K + noise I) V, matrix-free, entries recomputed from X (Sec. 2.1)."""
    X = _f64c(X)
    n, d = X.shape
    Vf = _f64f(V)
    c = Vf.shape[1]
    O = np.zeros((n, c), dtype=np.float64, order="F")
    if n and c:
        _load().or_kyv(_p(X), n, d, _p(_f64c(ell)), float(s2), float(noise), _p(Vf), n, c,
                       _p(O), n)
    return O[:, 0] if np.ndim(V) == 1 else O


def dkv(X, ell, s2, W) -> np.ndarray:
    """[dK/dlog l_1 W, ..., dK/dlog l_d W, dK/dlog s2 W] as a (d+1, n, c) array.

    dK_ij/dlog l_r = K_ij (x_ir - x_jr)^2 / l_r^2 and dK/dlog s2 = K, the
    derivatives of Eq. 1 that enter Eq. 2.
    """
    X = _f64c(X)
    n, d = X.shape
    Wf = _f64f(W)
    c = Wf.shape[1]
    G = np.zeros((d + 1) * n * c, dtype=np.float64)
    if n and c:
        _load().or_dkv(_p(X), n, d, _p(_f64c(ell)), float(s2), _p(Wf), n, c, _p(G))
    return G.reshape(d + 1, c, n).transpose(0, 2, 1)


def cholesky(A) -> np.ndarray:
    """Textbook lower Cholesky factor; raises ValueError if A is not SPD."""
    L = np.array(A, dtype=np.float64, order="C", copy=True)
    n = L.shape[0]
    st = _load().or_chol(_p(L), n)
    if st:
        raise ValueError(f"not positive definite at pivot {st - 1}")
    return L


def chol_solve(L, B) -> np.ndarray:
    """Solve (L L^T) X = B by forward and back substitution."""
    L = _f64c(L)
    Bf = np.array(_f64f(B), order="F", copy=True)
    n, c = Bf.shape
    _load().or_chol_solve(_p(L), n, _p(Bf), n, c)
    return Bf[:, 0] if np.ndim(B) == 1 else Bf


def dense_ky(X, ell, s2, noise) -> np.ndarray:
    K = gram(X, X, ell, s2)
    K[np.diag_indices_from(K)] += noise
    return K


def dense_solve(X, ell, s2, noise, B) -> np.ndarray:
    """alpha = K_y^{-1} B by Cholesky: the exact solution PCG converges to."""
    return chol_solve(cholesky(dense_ky(X, ell, s2, noise)), B)


def logml(X, ell, s2, noise, y) -> float:
    """log p(y|theta,X) = -1/2 log|K_y| - 1/2 y^T K_y^{-1} y - n/2 log 2pi (Sec. 2.1)."""
    L = cholesky(dense_ky(X, ell, s2, noise))
    a = chol_solve(L, y)
    n = L.shape[0]
    return float(-np.sum(np.log(np.diag(L))) - 0.5 * np.dot(y, a) - 0.5 * n * np.log(2 * np.pi))


# ---------------------------------------------------------------------------
# Preconditioners (Sec. 3)
# ---------------------------------------------------------------------------
class Nystrom:
    """P = K_XU K_UU^{-1} K_UX + noise I (Sec. 3.1), applied by the inversion lemma
    P^{-1} = noise^{-1} [I - K_XU (noise K_UU + K_UX K_XU)^{-1} K_UX]."""

    kind = 1

    def __init__(self, X, ell, s2, noise, idx):
        X = _f64c(X)
        self.n, d = X.shape
        self.idx = np.ascontiguousarray(idx, dtype=np.int64)
        self.m = int(self.idx.shape[0])
        self.noise = float(noise)
        self.KXU = np.empty((self.n, self.m), dtype=np.float64)
        self.LM = np.empty((self.m, self.m), dtype=np.float64)
        jit = ctypes.c_double(0.0)
        st = _load().or_nys_setup(_p(X), self.n, d, _p(_f64c(ell)), float(s2), self.noise,
                                  self.idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  self.m, _p(self.KXU), _p(self.LM), ctypes.byref(jit))
        if st:
            raise ValueError("Nystrom inner matrix not positive definite after jitter")
        self.jitter = jit.value

    def apply(self, R) -> np.ndarray:
        Rf = _f64f(R)
        Z = np.zeros_like(Rf, order="F")
        _load().or_nys_apply(self.n, self.m, self.noise, _p(self.KXU), _p(self.LM), _p(Rf),
                             self.n, Rf.shape[1], _p(Z), self.n)
        return Z[:, 0] if np.ndim(R) == 1 else Z


class BlockJacobi:
    """P = bldiag(K_y) over contiguous blocks of b rows (Sec. 3.3.1)."""

    kind = 2

    def __init__(self, X, ell, s2, noise, b):
        X = _f64c(X)
        self.n, d = X.shape
        self.b = int(b)
        nb = (self.n + self.b - 1) // self.b
        self.L = np.zeros(nb * self.b * self.b, dtype=np.float64)
        st = _load().or_bj_setup(_p(X), self.n, d, _p(_f64c(ell)), float(s2), float(noise),
                                 self.b, _p(self.L))
        if st:
            raise ValueError(f"block of K_y not positive definite near row {st - 1}")

    def apply(self, R) -> np.ndarray:
        Rf = _f64f(R)
        Z = np.zeros_like(Rf, order="F")
        _load().or_bj_apply(self.n, self.b, _p(self.L), _p(Rf), self.n, Rf.shape[1], _p(Z),
                            self.n)
        return Z[:, 0] if np.ndim(R) == 1 else Z


def pcg(X, ell, s2, noise, B, *, precond=None, tol=1e-8, tol_mode=0, max_iter=100000, X0=None,
        history=False):
    """Algorithm 1 (textbook form) on each column of B.

    Returns (Xsol, iters, relres, rc): iters per column (-1 = breakdown),
    relres = recomputed ||b - K_y x|| / ||b||, rc 0 ok / 1 max_iter / 2 breakdown.
    With history=True a fifth item holds the first column's recursive
    relative residual before each iteration.
    """
    Xd = _f64c(X)
    n, d = Xd.shape
    Bf = _f64f(B)
    c = Bf.shape[1]
    out = np.zeros((n, c), dtype=np.float64, order="F")
    iters = (ctypes.c_int * c)()
    rel = np.zeros(c, dtype=np.float64)
    X0f = _f64f(X0) if X0 is not None else None
    kind = 0 if precond is None else precond.kind
    KXU = precond.KXU if kind == 1 else None
    LM = precond.LM if kind == 1 else None
    Lbj = precond.L if kind == 2 else None
    m = precond.m if kind == 1 else 0
    b = precond.b if kind == 2 else 0
    nul = ctypes.cast(None, _d)
    hist = np.full(max_iter + 1, np.nan) if history else None
    rc = _load().or_pcg(_p(Xd), n, d, _p(_f64c(ell)), float(s2), float(noise), kind,
                        _p(KXU) if KXU is not None else nul, _p(LM) if LM is not None else nul, m,
                        _p(Lbj) if Lbj is not None else nul, b, _p(Bf), n, c, float(tol),
                        int(tol_mode), int(max_iter), _p(X0f) if X0f is not None else nul,
                        _p(out), n, iters, _p(rel), _p(hist) if history else nul)
    it = np.array(list(iters), dtype=np.int64)
    sol = out[:, 0] if np.ndim(B) == 1 else out
    if history:
        return sol, it, rel, int(rc), hist[: max(int(it[0]), 0) + 1]
    return sol, it, rel, int(rc)


# ---------------------------------------------------------------------------
# Gradient of the log marginal likelihood (Eq. 2) and its stochastic form
# ---------------------------------------------------------------------------
def _chain_iso(g_ard: np.ndarray, d: int, ard: bool) -> np.ndarray:
    """Isotropic kernel: d/dlog l = sum_r d/dlog l_r (all l_r tied)."""
    if ard:
        return g_ard
    return np.concatenate([[g_ard[:d].sum()], g_ard[d:]])


def grad_exact(X, log_theta, noise, y, ard=True) -> np.ndarray:
    """Eq. 2 with the exact trace: g_i = -1/2 tr(K_y^{-1} dK_y) + 1/2 a^T dK_y a.

    Dense, O(n^3): small n only.  Returns [d/dlog l_r..., d/dlog s2, d/dlog noise].
    """
    Xd = _f64c(X)
    n, d = Xd.shape
    ell, s2 = split_theta(log_theta, d, ard)
    L = cholesky(dense_ky(Xd, ell, s2, noise))
    Kinv = chol_solve(L, np.eye(n))
    a = chol_solve(L, y)
    K = gram(Xd, Xd, ell, s2)
    g = np.empty(d + 2)
    for r in range(d):
        diff2 = ((Xd[:, None, r] - Xd[None, :, r]) / ell[r]) ** 2
        dK = K * diff2
        g[r] = -0.5 * np.sum(Kinv * dK) + 0.5 * a @ dK @ a
    g[d] = -0.5 * np.sum(Kinv * K) + 0.5 * a @ K @ a
    g[d + 1] = -0.5 * noise * np.trace(Kinv) + 0.5 * noise * (a @ a)
    return _chain_iso(g, d, ard)


def grad_stochastic(X, log_theta, noise, y, probes, ard=True, solve=None) -> np.ndarray:
    """Eq. 2 with the trace replaced by the Rademacher estimate of Sec. 2.1:

    tr(K_y^{-1} dK_y) ~ (1/t) sum_k r_k^T K_y^{-1} dK_y r_k = (1/t) sum_k w_k^T (dK_y r_k),
    w_k = K_y^{-1} r_k (K_y^{-1} is symmetric).  ``solve(B)`` returns K_y^{-1} B;
    by default a dense Cholesky solve.
    """
    Xd = _f64c(X)
    n, d = Xd.shape
    ell, s2 = split_theta(log_theta, d, ard)
    R = _f64f(probes)
    t = R.shape[1]
    Bblk = np.asfortranarray(np.column_stack([np.asarray(y, dtype=np.float64), R]))
    if solve is None:
        S = dense_solve(Xd, ell, s2, noise, Bblk)
    else:
        S = solve(Bblk)
    a = S[:, 0]
    Wt = S[:, 1:]
    G = dkv(Xd, ell, s2, np.column_stack([a, R]))  # (d+1, n, 1+t)
    g = np.empty(d + 2)
    for q in range(d + 1):
        quad = a @ G[q][:, 0]
        tr = np.mean(np.sum(Wt * G[q][:, 1:], axis=0)) if t else 0.0
        g[q] = -0.5 * tr + 0.5 * quad
    trn = np.mean(np.sum(Wt * R, axis=0)) if t else 0.0
    g[d + 1] = -0.5 * noise * trn + 0.5 * noise * (a @ a)
    return _chain_iso(g, d, ard)


# ---------------------------------------------------------------------------
# Predictions (Sec. 2.1: the predictive mean and variance at test inputs; the
# variance needs one linear system per test point; Sec. 5 scores both)
# ---------------------------------------------------------------------------
def predict(X, ell, s2, noise, alpha, Xs, var=True):
    """Predictive mean m_* = K(X_*, X) alpha and latent variance
    v_* = s2 - k_*^T K_y^{-1} k_* (k_* = K(X, x_*)), by dense FP64 algebra.
    Add the noise to v_* for the predictive variance of a noisy target."""
    Ks = gram(Xs, X, ell, s2)  # (ns, n)
    mean = Ks @ np.asarray(alpha, dtype=np.float64)
    if not var:
        return mean, None
    W = dense_solve(X, ell, s2, noise, np.asfortranarray(Ks.T))  # K_y^{-1} k_* per column
    v = s2 - np.einsum("ij,ji->i", Ks, W)
    return mean, v


# ---------------------------------------------------------------------------
# FITC preconditioner (Sec. 3.1): P = Q + diag(K - Q) + noise I, Q = K_XU K_UU^{-1} K_UX
# ---------------------------------------------------------------------------
class FITC:
    """Dense FP64 construction of the FITC approximation of K_y (small n)."""

    kind = 3

    def __init__(self, X, ell, s2, noise, idx):
        X = _f64c(X)
        self.idx = np.ascontiguousarray(idx, dtype=np.int64)
        U = X[self.idx]
        KXU = gram(X, U, ell, s2)
        KUU = gram(U, U, ell, s2)
        Q = KXU @ chol_solve(cholesky(KUU), np.asfortranarray(KXU.T))
        diagK = np.full(X.shape[0], float(s2))  # K_ii = s2 (Eq. 1)
        self.P = Q - np.diag(np.diag(Q)) + np.diag(diagK + float(noise))
        self.L = cholesky(self.P)
        self.n = X.shape[0]

    def apply(self, R) -> np.ndarray:
        return chol_solve(self.L, R)


def pcg_dense(A, b, apply_pinv, tol=1e-8, tol_mode=0, max_iter=100000):
    """Textbook preconditioned CG (Algorithm 1 as read by the C oracle: when the
    recursive residual passes, the true one is recomputed and CG restarts from
    x, at most 5 times) on a dense SPD A, one right-hand side; returns
    (x, iterations).  Used with preconditioners the C oracle does not have."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n)
    thr = n * tol if tol_mode == 1 else tol * tol * (b @ b)
    it = 0
    for _restart in range(7):
        r = b - A @ x
        if r @ r <= thr or it >= max_iter or _restart == 6:
            break
        z = apply_pinv(r)
        p = z.copy()
        rho = r @ z
        while it < max_iter:
            q = A @ p
            a = rho / (p @ q)
            it += 1
            x += a * p
            r -= a * q
            if r @ r <= thr:
                break
            z = apply_pinv(r)
            rho_new = r @ z
            p = z + (rho_new / rho) * p
            rho = rho_new
    return x, it


# ---------------------------------------------------------------------------
# Spectral preconditioner (Sec. 3.2, random Fourier features)
# ---------------------------------------------------------------------------
class Spectral:
    """P = Phi Phi^T + noise I with the random-feature approximation of Sec. 3.2:
    K^_ij = (s2/m) sum_r cos(2 pi s_r^T (x_i - x_j)), written as Phi Phi^T with
    Phi_i = sqrt(s2/m) [cos(2 pi s_r^T x_i), sin(2 pi s_r^T x_i)]_{r=1..m} (the
    cosine of a difference is cos cos + sin sin).  The frequencies are drawn from
    N(0, Lambda / (4 pi^2)), Lambda = diag(1/l_r^2); they enter as standard-normal
    draws omega (m x d), s_r = omega_r / (2 pi l).  Dense FP64 (small n): P is
    formed and factored."""

    kind = 4

    def __init__(self, X, ell, s2, noise, omega):
        X = _f64c(X)
        n, d = X.shape
        omega = np.asarray(omega, dtype=np.float64).reshape(-1, d)
        m = omega.shape[0]
        ell = np.broadcast_to(np.asarray(ell, dtype=np.float64), (d,))
        S = omega / (2.0 * np.pi * ell[None, :])  # spectral points s_r (rows)
        ph = 2.0 * np.pi * (X @ S.T)              # n x m phases
        self.Phi = np.sqrt(float(s2) / m) * np.concatenate([np.cos(ph), np.sin(ph)], axis=1)
        self.Khat = self.Phi @ self.Phi.T
        self.P = self.Khat + float(noise) * np.eye(n)
        self.L = cholesky(self.P)
        self.n, self.m, self.noise = n, m, float(noise)

    def apply(self, R) -> np.ndarray:
        return chol_solve(self.L, R)


# ---------------------------------------------------------------------------
# GP classification: Laplace approximation with the probit likelihood
# (Sec. 2.2 and Appendix B)
# ---------------------------------------------------------------------------
def probit_terms(y, f):
    """Per point: log p(y_i|f_i) = log Phi(y_i f_i) (the probit likelihood of
    Appendix B), its first derivative g_i and W_ii = -(second derivative).
    With z = y f and r = N(z)/Phi(z): g = y r, W = r^2 + z r (y = +-1).  The
    ratio is taken through the log CDF so that it stays finite for z << 0."""
    from scipy.special import log_ndtr

    y = np.asarray(y, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    z = y * f
    lp = log_ndtr(z)
    r = np.exp(-0.5 * z * z - 0.5 * np.log(2.0 * np.pi) - lp)
    return lp, y * r, r * r + z * r


def laplace_probit(X, ell, s2, y, tol=1e-12, max_newton=100):
    """The Newton iteration for the posterior mode f^ of the Laplace
    approximation (Appendix B, Algorithm "Laplace approximation for GPs"), dense
    FP64 for small n.  Each step: W and g at f; b = W f + g; v = W^1/2 K b;
    solve B z = v with B = I + W^1/2 K W^1/2 (Cholesky here, PCG on the GPU);
    a = b - W^1/2 z; f = K a.  The paper only says "until convergence": the
    loop stops once the objective Psi(f) = log p(y|f) - 1/2 f^T K^{-1} f
    (= log p(y|f) - 1/2 a^T f) changes by at most tol * max(1, |Psi|), or after
    max_newton steps.  Returns f^, a, the step count, Psi and the approximate
    log marginal likelihood log q = -1/2 log|B| - 1/2 a^T f^ + log p(y|f^)
    (Sec. 2.2), with B taken at f^."""
    X = _f64c(X)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    K = gram(X, X, ell, s2)
    f = np.zeros(n)
    a = np.zeros(n)
    psi_old = float(probit_terms(y, f)[0].sum())
    psi = psi_old
    steps = 0
    while steps < max_newton:
        steps += 1
        _lp, g, W = probit_terms(y, f)
        sW = np.sqrt(W)
        b = W * f + g
        v = sW * (K @ b)
        B = np.eye(n) + sW[:, None] * K * sW[None, :]
        z = chol_solve(cholesky(B), v)
        a = b - sW * z
        f = K @ a
        psi = float(probit_terms(y, f)[0].sum() - 0.5 * a @ f)
        done = abs(psi - psi_old) <= tol * max(1.0, abs(psi))
        psi_old = psi
        if done:
            break
    lp, _g, W = probit_terms(y, f)
    sW = np.sqrt(W)
    LB = cholesky(np.eye(n) + sW[:, None] * K * sW[None, :])
    logq = float(-np.sum(np.log(np.diag(LB))) - 0.5 * a @ f + lp.sum())
    return {"f": f, "a": a, "steps": steps, "psi": psi, "logq": logq}


def laplace_predict(X, ell, s2, y, f, a, Xs):
    """Predictions of the probit classifier at test inputs Xs (Sec. 2.2 and
    Appendix B, "Prediction"): latent mean m_* = k_*^T a, latent variance
    v_* = s2 - k_*^T W^1/2 B^{-1} W^1/2 k_* (one B-solve per test point, B and W
    at the mode f), and the predictive probability Phi(m_* / sqrt(1 + v_*)),
    the exact Gaussian integral of the probit likelihood.  Dense FP64."""
    from scipy.special import ndtr

    X = _f64c(X)
    Ks = gram(Xs, X, ell, s2)  # (ns, n)
    mean = Ks @ np.asarray(a, dtype=np.float64)
    _lp, _g, W = probit_terms(y, f)
    sW = np.sqrt(W)
    K = gram(X, X, ell, s2)
    n = X.shape[0]
    LB = cholesky(np.eye(n) + sW[:, None] * K * sW[None, :])
    R = np.asfortranarray(sW[:, None] * Ks.T)
    V = chol_solve(LB, R)
    var = float(s2) - np.einsum("ij,ij->j", R, V)
    return mean, var, ndtr(mean / np.sqrt(1.0 + var))


# ---------------------------------------------------------------------------
# PITC preconditioner (Sec. 3.1): P = Q + bldiag(K - Q) + noise I
# ---------------------------------------------------------------------------
class PITC:
    """Dense FP64 construction of the PITC approximation of K_y (small n): the
    Nystrom Q = K_XU K_UU^{-1} K_UX off the diagonal blocks, K_y itself on the
    diagonal blocks (contiguous blocks of b rows in input order, the last one
    shorter), factored by Cholesky."""

    kind = 5

    def __init__(self, X, ell, s2, noise, idx, b):
        X = _f64c(X)
        n = X.shape[0]
        self.idx = np.ascontiguousarray(idx, dtype=np.int64)
        U = X[self.idx]
        KXU = gram(X, U, ell, s2)
        KUU = gram(U, U, ell, s2)
        Q = KXU @ chol_solve(cholesky(KUU), np.asfortranarray(KXU.T))
        K = gram(X, X, ell, s2)
        P = Q.copy()
        for r0 in range(0, n, int(b)):
            r1 = min(n, r0 + int(b))
            P[r0:r1, r0:r1] = K[r0:r1, r0:r1]
        P[np.diag_indices(n)] += float(noise)
        self.P = P
        self.L = cholesky(P)
        self.n, self.b = n, int(b)

    def apply(self, R) -> np.ndarray:
        return chol_solve(self.L, R)
