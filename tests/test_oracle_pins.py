"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these tests retypes the oracle's formula and compares it with itself:
each pin is a closed form, an invariant the paper states, a special case that
reduces to a library routine (SciPy / LAPACK), a finite-difference check, or
brute force on tiny inputs.  Each is chosen so that a plausible slip in the
oracle (a dropped term, a sign, a wrong index) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.spatial.distance import cdist

import oracle
import synthetic


def _lib_gram(X, Z, ell, s2):
    """RBF Gram matrix from SciPy's squared-Euclidean distance (Eq. 1)."""
    Xs = np.asarray(X, np.float64) / ell
    Zs = np.asarray(Z, np.float64) / ell
    return s2 * np.exp(-0.5 * cdist(Xs, Zs, "sqeuclidean"))


def _small(n=40, d=3, seed=0, ell=0.8, s2=1.3, noise=0.05):
    g = synthetic.rng(seed)
    X = g.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    ls = np.full(d, ell) * np.exp(0.2 * g.standard_normal(d))
    y = g.standard_normal(n)
    return X, ls, s2, noise, y


# --------------------------------------------------------------------- Eq. 1
def test_entry_closed_forms():
    # d = 1: |x - x'| = 1, l = 1 -> exp(-1/2); l = 2 and |x - x'| = 2 -> exp(-1/2)
    K = oracle.gram(np.array([[0.0]]), np.array([[1.0]]), np.array([1.0]), 1.0)
    assert K[0, 0] == pytest.approx(math.exp(-0.5), rel=1e-15)
    K = oracle.gram(np.array([[0.0]]), np.array([[2.0]]), np.array([2.0]), 3.0)
    assert K[0, 0] == pytest.approx(3.0 * math.exp(-0.5), rel=1e-15)
    # d = 2 with different lengthscales: exponent -1/2 (1/0.5^2 + 4/4) = -2.5
    K = oracle.gram(np.array([[0.0, 0.0]]), np.array([[1.0, 2.0]]), np.array([0.5, 2.0]), 1.0)
    assert K[0, 0] == pytest.approx(math.exp(-2.5), rel=1e-15)


def test_entries_match_library_and_invariants():
    X, ell, s2, _, _ = _small(n=30, d=4)
    K = oracle.gram(X, X, ell, s2)
    np.testing.assert_allclose(K, _lib_gram(X, X, ell, s2), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(np.diag(K), s2, rtol=1e-15)
    np.testing.assert_array_equal(K, K.T)
    assert np.all(K > 0) and np.all(K <= s2 * (1 + 1e-15))
    # ARD with tied lengthscales equals the isotropic kernel
    iso = np.full(4, 0.7)
    np.testing.assert_allclose(oracle.gram(X, X, iso, s2), _lib_gram(X, X, 0.7, s2), rtol=1e-13)


def test_matvec_matches_dense_product():
    X, ell, s2, noise, _ = _small(n=57, d=5)
    V = synthetic.rng(3).standard_normal((57, 3))
    Ky = _lib_gram(X, X, ell, s2) + noise * np.eye(57)
    np.testing.assert_allclose(oracle.kyv(X, ell, s2, noise, V), Ky @ V, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.kyv(X, ell, s2, noise, V[:, 0]), Ky @ V[:, 0], rtol=1e-12,
                               atol=1e-12)


# --------------------------------------------------------- Cholesky / solve
def test_cholesky_and_solve_match_lapack():
    X, ell, s2, noise, y = _small(n=80, d=3)
    Ky = _lib_gram(X, X, ell, s2) + noise * np.eye(80)
    L = oracle.cholesky(Ky)
    np.testing.assert_allclose(L, np.linalg.cholesky(Ky), rtol=1e-10, atol=1e-12)
    B = np.column_stack([y, synthetic.rng(5).standard_normal(80)])
    np.testing.assert_allclose(oracle.chol_solve(L, B), sla.solve(Ky, B, assume_a="pos"),
                               rtol=1e-8, atol=1e-10)
    with pytest.raises(ValueError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_logml_matches_library():
    X, ell, s2, noise, y = _small(n=50, d=2)
    Ky = _lib_gram(X, X, ell, s2) + noise * np.eye(50)
    sign, ld = np.linalg.slogdet(Ky)
    ref = -0.5 * ld - 0.5 * y @ np.linalg.solve(Ky, y) - 25 * np.log(2 * np.pi)
    assert sign > 0
    assert oracle.logml(X, ell, s2, noise, y) == pytest.approx(ref, rel=1e-11)


# ------------------------------------------------------------- Algorithm 1
def test_cg_converges_within_n_and_matches_solve():
    # P = I, small well-conditioned system: exact arithmetic needs at most n
    # steps; in FP64 the n-th iterate is already at rounding level.
    g = synthetic.rng(11)
    X = g.standard_normal((16, 2))
    ell = np.full(2, 0.4)
    y = g.standard_normal(16)
    x, it, rel, rc = oracle.pcg(X, ell, 1.0, 0.1, y, tol=1e-8)
    assert rc == 0 and 0 < it[0] <= 16 and rel[0] <= 1e-8
    Ky = _lib_gram(X, X, ell, 1.0) + 0.1 * np.eye(16)
    np.testing.assert_allclose(x, sla.solve(Ky, y, assume_a="pos"), rtol=1e-8, atol=1e-10)


def _krylov_minimizer(A, Pinv, b, k):
    """argmin over K_k(Pinv A, Pinv b) of the A-norm error: the k-th (P)CG iterate."""
    v = Pinv @ b
    Q = np.zeros((len(b), 0))
    for _ in range(k):
        for _ in range(2):  # Gram-Schmidt with re-orthogonalisation
            v = v - Q @ (Q.T @ v)
        Q = np.column_stack([Q, v / np.linalg.norm(v)])
        v = Pinv @ (A @ Q[:, -1])
    c = np.linalg.solve(Q.T @ A @ Q, Q.T @ b)
    return Q @ c


@pytest.mark.parametrize("precond", ["none", "nystrom", "bj"])
def test_pcg_iterates_are_krylov_minimizers(precond):
    # The k-th PCG iterate minimizes ||x - x*||_A over the preconditioned
    # Krylov space; a wrong alpha, beta, sign or z/r mix-up breaks this.
    X, ell, s2, noise, y = _small(n=48, d=3, noise=0.05)
    A = _lib_gram(X, X, ell, s2) + noise * np.eye(48)
    if precond == "nystrom":
        P = oracle.Nystrom(X, ell, s2, noise, synthetic.inducing_subset(48, 6, 1))
        Pinv = P.apply(np.eye(48))
    elif precond == "bj":
        P = oracle.BlockJacobi(X, ell, s2, noise, 10)
        Pinv = P.apply(np.eye(48))
    else:
        P, Pinv = None, np.eye(48)
    for k in range(1, 6):
        xk, it, _, rc = oracle.pcg(X, ell, s2, noise, y, precond=P, tol=1e-15, max_iter=k)
        assert it[0] == k and rc == 1
        ref = _krylov_minimizer(A, Pinv, y, k)
        np.testing.assert_allclose(xk, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())


def test_cg_terminates_by_distinct_eigenvalue_count():
    # Three distinct points repeated: K has rank <= 3, so K_y has at most 4
    # distinct eigenvalues and CG (exact arithmetic) stops within 4 steps.
    # A wrong beta, sign or denominator in the recurrence breaks this.
    base = np.array([[0.0, 0.0], [0.7, -0.2], [-0.4, 1.1]])
    X = np.repeat(base, 20, axis=0)
    y = synthetic.rng(2).standard_normal(60)
    x, it, rel, rc = oracle.pcg(X, np.ones(2), 1.0, 0.3, y, tol=1e-11)
    assert rc == 0 and it[0] <= 4, it
    assert rel[0] <= 1e-11


def test_pcg_paper_absolute_stop_rule():
    X, ell, s2, noise, y = _small(n=60, d=3, noise=0.01)
    # ||r||^2 < n * 1e-10, the rule of Sec. 4
    x, it, rel, rc = oracle.pcg(X, ell, s2, noise, y, tol=1e-10, tol_mode=1)
    Ky = _lib_gram(X, X, ell, s2) + noise * np.eye(60)
    r = y - Ky @ x
    assert rc == 0 and r @ r < 60 * 1e-10


def test_pcg_zero_rhs_and_warm_start():
    X, ell, s2, noise, y = _small(n=40, d=3)
    B = np.column_stack([np.zeros(40), y])
    x, it, rel, rc = oracle.pcg(X, ell, s2, noise, B, tol=1e-10)
    assert it[0] == 0 and np.all(x[:, 0] == 0) and rel[0] == 0
    # starting from the solution needs no iteration
    x2, it2, _, _ = oracle.pcg(X, ell, s2, noise, y, tol=1e-8, X0=x[:, 1])
    assert it2[0] == 0


# ------------------------------------------------------- preconditioners
def test_nystrom_with_all_points_is_exact_one_step():
    # m = n: M = K (noise I + K), so P = K_y and PCG converges in one step.
    g = synthetic.rng(7)
    X = g.standard_normal((64, 8))
    ell = np.ones(8)
    y = g.standard_normal(64)
    P = oracle.Nystrom(X, ell, 1.0, 0.1, np.arange(64))
    x, it, rel, rc = oracle.pcg(X, ell, 1.0, 0.1, y, precond=P, tol=1e-10)
    assert rc == 0 and it[0] == 1, it
    assert rel[0] <= 1e-10


def test_nystrom_inverse_against_dense_P():
    X, ell, s2, noise, _ = _small(n=128, d=3, noise=0.02)
    idx = synthetic.inducing_subset(128, 16, seed=4)
    P = oracle.Nystrom(X, ell, s2, noise, idx)
    KXU = _lib_gram(X, X[idx], ell, s2)
    KUU = _lib_gram(X[idx], X[idx], ell, s2)
    Pd = KXU @ np.linalg.solve(KUU, KXU.T) + noise * np.eye(128)
    v = synthetic.rng(9).standard_normal((128, 2))
    np.testing.assert_allclose(P.apply(Pd @ v), v, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(P.apply(v), np.linalg.solve(Pd, v), rtol=1e-8, atol=1e-8)


def test_block_jacobi_inverse_and_full_block():
    X, ell, s2, noise, y = _small(n=100, d=3)
    Ky = _lib_gram(X, X, ell, s2) + noise * np.eye(100)
    b = 32  # blocks 32, 32, 32, 4 (ragged tail)
    Pd = np.zeros_like(Ky)
    for r0 in range(0, 100, b):
        sl = slice(r0, min(r0 + b, 100))
        Pd[sl, sl] = Ky[sl, sl]
    P = oracle.BlockJacobi(X, ell, s2, noise, b)
    v = synthetic.rng(1).standard_normal((100, 2))
    np.testing.assert_allclose(P.apply(v), np.linalg.solve(Pd, v), rtol=1e-9, atol=1e-9)
    # one block covering everything is P = K_y: one step
    Pfull = oracle.BlockJacobi(X, ell, s2, noise, 100)
    x, it, rel, rc = oracle.pcg(X, ell, s2, noise, y, precond=Pfull, tol=1e-10)
    assert rc == 0 and it[0] == 1


def test_preconditioned_system_is_spd():
    X, ell, s2, noise, _ = _small(n=96, d=3, noise=0.01)
    Ky = _lib_gram(X, X, ell, s2) + noise * np.eye(96)
    assert np.linalg.eigvalsh(Ky).min() >= noise * (1 - 1e-10)
    I = np.eye(96)
    for P in (oracle.Nystrom(X, ell, s2, noise, synthetic.inducing_subset(96, 10, 0)),
              oracle.BlockJacobi(X, ell, s2, noise, 24)):
        Pinv = P.apply(I)
        np.testing.assert_allclose(Pinv, Pinv.T, atol=1e-8 * np.abs(Pinv).max())
        ev = np.linalg.eigvals(Pinv @ Ky)
        assert np.abs(ev.imag).max() < 1e-6 * np.abs(ev.real).max()
        assert ev.real.min() > 0


# -------------------------------------------- Eq. 2 and the stochastic trace
def test_exact_gradient_matches_finite_differences():
    X, ell, s2, noise, y = _small(n=45, d=3, noise=0.07)
    lt = np.concatenate([np.log(ell), [np.log(s2)]])
    g = oracle.grad_exact(X, lt, noise, y, ard=True)
    h = 1e-5

    def lp(theta, lnoise):
        e, s = oracle.split_theta(theta, 3, True)
        return oracle.logml(X, e, s, math.exp(lnoise), y)

    fd = np.empty(5)
    for q in range(4):
        tp, tm = lt.copy(), lt.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (lp(tp, math.log(noise)) - lp(tm, math.log(noise))) / (2 * h)
    fd[4] = (lp(lt, math.log(noise) + h) - lp(lt, math.log(noise) - h)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7)


def test_isotropic_gradient_matches_finite_differences():
    X, _, s2, noise, y = _small(n=30, d=2, noise=0.05)
    lt = np.array([math.log(0.9), math.log(s2)])
    g = oracle.grad_exact(X, lt, noise, y, ard=False)
    h = 1e-5

    def lp(theta):
        e, s = oracle.split_theta(theta, 2, False)
        return oracle.logml(X, e, s, noise, y)

    fd = [(lp(lt + h * np.eye(2)[q]) - lp(lt - h * np.eye(2)[q])) / (2 * h) for q in range(2)]
    np.testing.assert_allclose(g[:2], fd, rtol=1e-6, atol=1e-7)


def test_dkv_matches_finite_differences_of_matvec():
    X, ell, s2, _, _ = _small(n=33, d=3)
    W = synthetic.rng(4).standard_normal((33, 2))
    G = oracle.dkv(X, ell, s2, W)
    h = 1e-6
    for r in range(3):
        ep, em = ell.copy(), ell.copy()
        ep[r] *= math.exp(h)
        em[r] *= math.exp(-h)
        fd = (oracle.kyv(X, ep, s2, 0.0, W) - oracle.kyv(X, em, s2, 0.0, W)) / (2 * h)
        np.testing.assert_allclose(G[r], fd, rtol=1e-7, atol=1e-9)
    fd = (oracle.kyv(X, ell, s2 * math.exp(h), 0.0, W)
          - oracle.kyv(X, ell, s2 * math.exp(-h), 0.0, W)) / (2 * h)
    np.testing.assert_allclose(G[3], fd, rtol=1e-7, atol=1e-9)


def test_hutchinson_over_all_sign_vectors_equals_exact_gradient():
    # E[r r^T] = I over Rademacher r: averaging over all 2^n sign vectors is
    # exactly the trace, so the stochastic gradient equals Eq. 2.
    n = 10
    X, ell, s2, noise, y = _small(n=n, d=2, noise=0.2)
    lt = np.concatenate([np.log(ell), [np.log(s2)]])
    R = np.array(list(itertools.product([-1.0, 1.0], repeat=n))).T
    gs = oracle.grad_stochastic(X, lt, noise, y, R, ard=True)
    ge = oracle.grad_exact(X, lt, noise, y, ard=True)
    np.testing.assert_allclose(gs, ge, rtol=1e-10, atol=1e-12)


def test_hutchinson_variance_closed_form():
    # Var(r^T A r) = sum_{i != j} A_ij (A_ij + A_ji) for Rademacher r.
    n = 8
    A = synthetic.rng(6).standard_normal((n, n))
    R = np.array(list(itertools.product([-1.0, 1.0], repeat=n)))
    q = np.einsum("ki,ij,kj->k", R, A, R)
    assert q.mean() == pytest.approx(np.trace(A), abs=1e-12)
    off = A * (A + A.T)
    np.fill_diagonal(off, 0.0)
    assert q.var() == pytest.approx(off.sum(), rel=1e-12)


def test_stochastic_gradient_with_pcg_solves_matches_dense():
    X, ell, s2, noise, y = _small(n=70, d=3, noise=0.03)
    lt = np.concatenate([np.log(ell), [np.log(s2)]])
    R = synthetic.rademacher(70, 5, seed=1)
    P = oracle.Nystrom(X, ell, s2, noise, synthetic.inducing_subset(70, 9, 2))

    def solve(B):
        return oracle.pcg(X, ell, s2, noise, B, precond=P, tol=1e-13)[0]

    np.testing.assert_allclose(oracle.grad_stochastic(X, lt, noise, y, R, solve=solve),
                               oracle.grad_stochastic(X, lt, noise, y, R), rtol=1e-8, atol=1e-9)


def test_synthetic_inputs_are_seeded():
    a = synthetic.config1(seed=0, n=256)
    b = synthetic.config1(seed=0, n=256)
    assert a.X.dtype == np.float32 and a.X.flags.c_contiguous
    np.testing.assert_array_equal(a.X, b.X)
    np.testing.assert_array_equal(a.y, b.y)
    R = synthetic.rademacher(100, 4, 3)
    assert set(np.unique(R)) == {-1.0, 1.0} and R.flags.f_contiguous
    idx = synthetic.inducing_subset(100, 10, 0)
    assert np.all(np.diff(idx) > 0) and idx.max() < 100


# ------------------------------------------------- warm-start network (MLP)
def _mlp_case():
    from oracle import mlp
    P = synthetic.mlp_init(3, 3, 5, 4, 2)
    for k in ("b1", "b2", "b3"):
        P[k] = synthetic.rng(9).standard_normal(P[k].shape) * 0.3
    X = synthetic.rng(1).standard_normal((4, 3))
    T = synthetic.rng(2).standard_normal((4, 2))
    return mlp, P, X, T


def test_mlp_backprop_matches_finite_differences():
    mlp, P, X, T = _mlp_case()
    g = mlp.backward(P, X, T)
    h = 1e-6
    for k in mlp.NAMES:
        fd = np.zeros_like(P[k])
        for idx in np.ndindex(P[k].shape):
            Pp = {q: v.copy() for q, v in P.items()}
            Pm = {q: v.copy() for q, v in P.items()}
            Pp[k][idx] += h
            Pm[k][idx] -= h
            fd[idx] = (mlp.loss(Pp, X, T) - mlp.loss(Pm, X, T)) / (2 * h)
        np.testing.assert_allclose(g[k], fd, rtol=1e-7, atol=1e-10)


def test_mlp_forward_closed_form_and_adam_first_step():
    mlp, P, X, T = _mlp_case()
    Z = {k: np.zeros_like(v) for k, v in P.items()}
    Z["b3"] = np.array([0.5, -2.0])
    out, _ = mlp.forward(Z, X)  # tanh(0) = 0: the output is the last bias
    np.testing.assert_array_equal(out, np.tile([0.5, -2.0], (4, 1)))
    # Adam, first step from zero moments: m^ = g, v^ = g^2, step = lr g/(|g| + eps)
    g = mlp.backward(P, X, T)
    P2 = mlp.adam_step({k: v.copy() for k, v in P.items()}, g, {}, lr=1e-2)
    for k in mlp.NAMES:
        np.testing.assert_allclose(P2[k] - P[k], -1e-2 * g[k] / (np.abs(g[k]) + 1e-8),
                                   rtol=1e-12, atol=1e-15)


# ----------------------------------------------------------------- predictions
def test_predict_single_training_point_closed_form():
    # n = 1: K_y = s2 + noise, so m_* = s2 e^{-q} y / (s2 + noise) and
    # v_* = s2 - s2^2 e^{-2q} / (s2 + noise) with q = |x - x_*|^2 / (2 l^2)
    X = np.array([[0.3, -0.2]], dtype=np.float32)
    Xs = np.array([[0.3, -0.2], [1.0, 0.5]], dtype=np.float32)
    ell, s2, noise, y = np.array([0.7, 1.3]), 1.7, 0.05, 2.0
    alpha = np.array([y / (s2 + noise)])
    m, v = oracle.predict(X, ell, s2, noise, alpha, Xs)
    d = (Xs.astype(np.float64) - X.astype(np.float64)) / ell
    e = np.exp(-0.5 * (d ** 2).sum(1))
    np.testing.assert_allclose(m, s2 * e * y / (s2 + noise), rtol=1e-14)
    np.testing.assert_allclose(v, s2 - (s2 * e) ** 2 / (s2 + noise), rtol=1e-13)
    assert v[0] == pytest.approx(s2 * noise / (s2 + noise), rel=1e-13)


def test_predict_far_point_and_interpolation():
    p = synthetic.make_problem(60, 3, 4, ell=0.8, noise=1e-8)
    ell, s2 = oracle.split_theta(p.log_theta, 3, True)
    alpha = oracle.dense_solve(p.X, ell, s2, p.noise, p.y[:, None])[:, 0]
    far = np.full((1, 3), 50.0, dtype=np.float32)
    m, v = oracle.predict(p.X, ell, s2, p.noise, alpha, np.vstack([p.X[:5], far]))
    # at training inputs with (almost) no noise the mean interpolates y and the
    # variance vanishes; far from the data the prior returns: m = 0, v = s2
    np.testing.assert_allclose(m[:5], p.y[:5], atol=1e-5)
    assert np.all(np.abs(v[:5]) <= 1e-5)
    assert abs(m[5]) <= 1e-12 and v[5] == pytest.approx(s2, rel=1e-12)


def test_predict_variance_bounds_and_monotone_in_data():
    p = synthetic.make_problem(80, 4, 6, ell=1.1, noise=0.05)
    ell, s2 = oracle.split_theta(p.log_theta, 4, True)
    Xs = synthetic.rng(7).standard_normal((40, 4)).astype(np.float32)
    a = oracle.dense_solve(p.X, ell, s2, p.noise, p.y[:, None])[:, 0]
    _, v = oracle.predict(p.X, ell, s2, p.noise, a, Xs)
    assert np.all(v > 0) and np.all(v <= s2 * (1 + 1e-12))
    # conditioning on fewer training points can only increase the variance
    a2 = oracle.dense_solve(p.X[:40], ell, s2, p.noise, p.y[:40, None])[:, 0]
    _, v2 = oracle.predict(p.X[:40], ell, s2, p.noise, a2, Xs)
    assert np.all(v2 >= v - 1e-12)


# -------------------------------------------------------------------- FITC
def test_fitc_diagonal_matches_k_y_and_is_spd():
    # FITC keeps the diagonal of K_y exactly (the correction diag(K - Q) puts
    # it back) and P - noise I = Q + diag(K - Q) is positive semi-definite
    p = synthetic.make_problem(120, 3, 9, ell=0.9, noise=0.02)
    ell, s2 = oracle.split_theta(p.log_theta, 3, True)
    idx = synthetic.inducing_subset(120, 15, seed=2)
    F = oracle.FITC(p.X, ell, s2, p.noise, idx)
    np.testing.assert_allclose(np.diag(F.P), s2 + p.noise, rtol=1e-14)
    w = np.linalg.eigvalsh(F.P - p.noise * np.eye(120))
    assert w.min() >= -1e-10 * w.max()
    # off the diagonal it is the Nystrom approximation, not K
    K = oracle.gram(p.X, p.X, ell, s2)
    assert np.abs(F.P - K - p.noise * np.eye(120)).max() > 1e-3


def test_fitc_with_all_points_is_k_y():
    # m = n: Q = K, diag(K - Q) = 0, P = K + noise I; PCG then converges at once
    p = synthetic.make_problem(50, 2, 3, ell=1.0, noise=0.1)
    ell, s2 = oracle.split_theta(p.log_theta, 2, True)
    F = oracle.FITC(p.X, ell, s2, p.noise, np.arange(50))
    Ky = oracle.dense_ky(p.X, ell, s2, p.noise)
    np.testing.assert_allclose(F.P, Ky, atol=1e-8 * np.abs(Ky).max())
    _, it = oracle.pcg_dense(Ky, p.y, F.apply, tol=1e-10)
    assert it == 1


def test_pcg_dense_matches_c_oracle_iterations():
    # the NumPy PCG used with FITC follows the same recurrence as the C oracle
    p = synthetic.make_problem(200, 4, 12, ell=1.3, noise=0.01)
    ell, s2 = oracle.split_theta(p.log_theta, 4, True)
    Ky = oracle.dense_ky(p.X, ell, s2, p.noise)
    idx = synthetic.inducing_subset(200, 20, seed=4)
    N = oracle.Nystrom(p.X, ell, s2, p.noise, idx)
    for pc in (None, N):
        _, it_c, _, _ = oracle.pcg(p.X, ell, s2, p.noise, p.y, precond=pc, tol=1e-9)
        x, it_d = oracle.pcg_dense(Ky, p.y, (pc.apply if pc else (lambda r: r)), tol=1e-9)
        # same recurrence and restart rule; rounding order differs (dense product)
        assert abs(int(it_c[0]) - it_d) <= max(2, 0.05 * int(it_c[0])), (int(it_c[0]), it_d)
        assert np.linalg.norm(Ky @ x - p.y) <= 1e-9 * np.linalg.norm(p.y)


# ------------------------------------------------- Sec. 3.2 spectral features
def test_spectral_diagonal_rank_and_shift_invariance():
    # cos^2 + sin^2 = 1 puts s2 on the diagonal for any draws; the features
    # depend on x_i - x_j only; Phi has 2m columns, so rank(K^) <= 2m
    X, ls, s2, noise, _ = _small(30, 3, seed=4)
    om = synthetic.spectral_draws(25, 3, seed=5)
    S = oracle.Spectral(X, ls, s2, noise, om)
    np.testing.assert_allclose(np.diag(S.Khat), s2, rtol=1e-13)
    S2 = oracle.Spectral(X + np.array([0.7, -1.9, 3.1]), ls, s2, noise, om)
    np.testing.assert_allclose(S2.Khat, S.Khat, atol=1e-12 * s2)
    S3 = oracle.Spectral(X, ls, s2, noise, om[:5])
    w = np.linalg.eigvalsh(S3.Khat)
    assert (w > 1e-10 * w.max()).sum() <= 10


def test_spectral_converges_to_the_rbf_kernel():
    # E cos(w^T (x - x') / l) = exp(-|(x - x') / l|^2 / 2) for w ~ N(0, I), the
    # spectral density of Eq. 1: with m draws each entry has a standard error of
    # at most s2 / sqrt(2m); a slip in the 2 pi or 1/l scaling is off by O(1)
    X, ls, s2, noise, _ = _small(25, 3, seed=6)
    m = 40000
    S = oracle.Spectral(X, ls, s2, noise, synthetic.spectral_draws(m, 3, seed=7))
    K = _lib_gram(X, X, ls, s2)
    assert np.abs(S.Khat - K).max() <= 6.0 * s2 / math.sqrt(2 * m)


def test_spectral_inversion_lemma_carries_the_noise():
    # (Phi Phi^T + lam I)^{-1} v = lam^{-1} [v - Phi (lam I + Phi^T Phi)^{-1} Phi^T v]
    # (the inversion lemma); the printed (I + Phi^T Phi) holds only for lam = 1
    X, ls, s2, _, _ = _small(40, 3, seed=8)
    lam = 0.05
    S = oracle.Spectral(X, ls, s2, lam, synthetic.spectral_draws(12, 3, seed=9))
    v = synthetic.rng(10).standard_normal(40)
    F = S.Phi
    I2 = np.eye(F.shape[1])
    lemma = (v - F @ np.linalg.solve(lam * I2 + F.T @ F, F.T @ v)) / lam
    np.testing.assert_allclose(S.apply(v), lemma, rtol=1e-9, atol=1e-9 * np.abs(lemma).max())
    printed = (v - F @ np.linalg.solve(I2 + F.T @ F, F.T @ v)) / lam
    assert np.linalg.norm(printed - lemma) > 1e-3 * np.linalg.norm(lemma)


# ------------------------------------- App. B: probit likelihood and Laplace
def test_probit_terms_closed_form_and_finite_differences():
    from scipy.stats import norm

    y = np.array([1.0, -1.0, 1.0, -1.0])
    lp, g, W = oracle.probit_terms(y, np.zeros(4))
    np.testing.assert_allclose(lp, -math.log(2.0), rtol=1e-15)
    np.testing.assert_allclose(g, y * math.sqrt(2.0 / math.pi), rtol=1e-14)
    np.testing.assert_allclose(W, 2.0 / math.pi, rtol=1e-14)
    # derivatives of log Phi(y f) by central differences of SciPy's log CDF
    y = np.array([1.0, -1.0, 1.0, -1.0, 1.0, -1.0])
    f = np.array([-7.0, -0.3, 0.4, 6.5, -25.0, 2.2])
    lp, g, W = oracle.probit_terms(y, f)
    L = lambda ff: norm.logcdf(y * ff)  # noqa: E731
    np.testing.assert_allclose(lp, L(f), rtol=1e-13)
    h = 1e-5
    np.testing.assert_allclose(g, (L(f + h) - L(f - h)) / (2 * h), rtol=1e-7)
    h = 1e-3
    np.testing.assert_allclose(W, -(L(f + h) - 2 * L(f) + L(f - h)) / h**2, rtol=1e-5)
    assert np.all((W > 0.0) & (W < 1.0))


def _laplace_small(n, d, seed, s2=2.0, ell=0.9):
    p = synthetic.classification_problem(n, d, seed, s2=s2, ell=ell)
    ls, s2 = oracle.split_theta(p.log_theta, d, True)
    return p, ls, s2


def test_laplace_mode_is_stationary():
    # at the mode grad Psi = g(f^) - K^{-1} f^ = 0, so f^ = K g(f^) and a = K^{-1} f^
    # = g(f^); Newton on the concave Psi converges in a handful of steps
    p, ls, s2 = _laplace_small(80, 3, seed=3)
    r = oracle.laplace_probit(p.X, ls, s2, p.y)
    K = _lib_gram(p.X, p.X, ls, s2)
    _, g, _ = oracle.probit_terms(p.y, r["f"])
    assert np.linalg.norm(K @ g - r["f"]) <= 1e-8 * np.linalg.norm(r["f"])
    assert np.linalg.norm(r["a"] - g) <= 1e-6 * np.linalg.norm(g)
    assert 3 <= r["steps"] <= 12
    # the labels are explained: sign(f^) agrees with most of them
    assert np.mean(np.sign(r["f"]) == p.y) > 0.8


def test_laplace_mode_matches_a_generic_optimiser():
    # maximise Psi(f) = sum log Phi(y f) - 1/2 f^T K^{-1} f with SciPy's BFGS in
    # the whitened variable f = L u (L L^T = K + tiny jitter), log CDF from SciPy
    from scipy.optimize import minimize
    from scipy.stats import norm

    p, ls, s2 = _laplace_small(14, 2, seed=5)
    K = _lib_gram(p.X, p.X, ls, s2)
    Lk = np.linalg.cholesky(K + 1e-10 * np.eye(14))
    y = p.y

    def negpsi(u):
        f = Lk @ u
        z = y * f
        ratio = np.exp(norm.logpdf(z) - norm.logcdf(z))
        return -(norm.logcdf(z).sum() - 0.5 * u @ u), -(Lk.T @ (y * ratio) - u)

    res = minimize(negpsi, np.zeros(14), jac=True, method="BFGS",
                   options={"gtol": 1e-11, "maxiter": 10000})
    f_ref = Lk @ res.x
    r = oracle.laplace_probit(p.X, ls, s2, y)
    np.testing.assert_allclose(r["f"], f_ref, rtol=1e-5, atol=1e-6 * np.abs(f_ref).max())


def test_laplace_log_marginal_is_the_gaussian_integral_form():
    # the Laplace approximation of log int p(y|f) N(f|0,K) df is
    # log p(y|f^) + log N(f^|0,K) + n/2 log 2 pi - 1/2 log|K^{-1} + W|; Sec. 2.2's
    # -1/2 log|B| - 1/2 f^T K^{-1} f + log p(y|f^) must equal it
    p, ls, s2 = _laplace_small(30, 3, seed=7, ell=0.6)
    r = oracle.laplace_probit(p.X, ls, s2, p.y)
    K = _lib_gram(p.X, p.X, ls, s2)
    f = r["f"]
    lp, _, W = oracle.probit_terms(p.y, f)
    Kinv = np.linalg.inv(K)
    n = 30
    lognorm = -0.5 * f @ Kinv @ f - 0.5 * np.linalg.slogdet(K)[1] - 0.5 * n * math.log(2 * math.pi)
    ref = lp.sum() + lognorm + 0.5 * n * math.log(2 * math.pi) \
        - 0.5 * np.linalg.slogdet(Kinv + np.diag(W))[1]
    assert r["logq"] == pytest.approx(ref, rel=1e-7)


def test_laplace_one_point_closed_form():
    # n = 1, K = s2: the mode is the root of f - s2 g(f) = 0, and
    # log q = log Phi(y f) - f^2 / (2 s2) - 1/2 log(1 + s2 W)
    from scipy.optimize import brentq
    from scipy.stats import norm

    for y, s2 in ((1.0, 3.0), (-1.0, 0.4)):
        gfun = lambda f: y * norm.pdf(f) / norm.cdf(y * f)  # noqa: E731
        f = brentq(lambda f: f - s2 * gfun(f), -10.0, 10.0, xtol=1e-15)
        z = y * f
        rr = norm.pdf(z) / norm.cdf(z)
        Wv = rr * rr + z * rr
        ref = math.log(norm.cdf(z)) - f * f / (2 * s2) - 0.5 * math.log(1 + s2 * Wv)
        r = oracle.laplace_probit(np.zeros((1, 1), np.float32), np.ones(1), s2, np.array([y]))
        assert r["f"][0] == pytest.approx(f, rel=1e-10)
        assert r["logq"] == pytest.approx(ref, rel=1e-10)


def test_laplace_predictive_variance_is_the_posterior_form():
    # s2 - k^T W^1/2 B^{-1} W^1/2 k = s2 - k^T (K + W^{-1})^{-1} k (the inversion
    # lemma; the Gaussian posterior of the latent at x_*), computed with NumPy
    p, ls, s2 = _laplace_small(40, 3, seed=9, ell=0.8)
    r = oracle.laplace_probit(p.X, ls, s2, p.y)
    Xs = synthetic.rng(3).standard_normal((7, 3))
    m, v, pr = oracle.laplace_predict(p.X, ls, s2, p.y, r["f"], r["a"], Xs)
    K = _lib_gram(p.X, p.X, ls, s2)
    ks = _lib_gram(p.X, Xs, ls, s2)  # (n, ns)
    _, g, W = oracle.probit_terms(p.y, r["f"])
    v_ref = s2 - np.einsum("ij,ij->j", ks, np.linalg.solve(K + np.diag(1.0 / W), ks))
    np.testing.assert_allclose(v, v_ref, rtol=1e-8)
    np.testing.assert_allclose(m, ks.T @ g, rtol=1e-6, atol=1e-9)
    assert np.all((v > 0) & (v <= s2)) and np.all((pr > 0) & (pr < 1))


def test_laplace_predictive_probability_is_the_gaussian_integral():
    # Phi(m / sqrt(1 + v)) = int Phi(t) N(t | m, v) dt, checked by quadrature; far
    # from the data the prediction falls back to the prior (m = 0, v = s2, 1/2)
    from scipy.integrate import quad
    from scipy.stats import norm

    p, ls, s2 = _laplace_small(30, 2, seed=11, ell=0.7)
    r = oracle.laplace_probit(p.X, ls, s2, p.y)
    Xs = np.array([[0.3, -0.2], [1.1, 0.4], [60.0, -80.0]])
    m, v, pr = oracle.laplace_predict(p.X, ls, s2, p.y, r["f"], r["a"], Xs)
    for k in range(2):
        ref, _ = quad(lambda t: norm.cdf(t) * norm.pdf(t, m[k], math.sqrt(v[k])),
                      m[k] - 12 * math.sqrt(v[k]), m[k] + 12 * math.sqrt(v[k]),
                      epsabs=1e-13, epsrel=1e-12)
        assert pr[k] == pytest.approx(ref, rel=1e-9)
    assert abs(m[2]) < 1e-12 and v[2] == pytest.approx(s2, rel=1e-12)
    assert pr[2] == pytest.approx(0.5, abs=1e-12)


def test_laplace_prediction_one_point_closed_form():
    # n = 1, x_* = x_1: m = s2 a, v = s2 - s2^2 W / (1 + s2 W) = s2 / (1 + s2 W)
    X = np.zeros((1, 2), np.float32)
    for y, s2 in ((1.0, 2.5), (-1.0, 0.7)):
        r = oracle.laplace_probit(X, np.ones(2), s2, np.array([y]))
        _, _, W = oracle.probit_terms(np.array([y]), r["f"])
        m, v, _ = oracle.laplace_predict(X, np.ones(2), s2, np.array([y]), r["f"], r["a"], X)
        assert m[0] == pytest.approx(s2 * r["a"][0], rel=1e-13)
        assert v[0] == pytest.approx(s2 / (1 + s2 * W[0]), rel=1e-12)


# ------------------------------------------------------------- Sec. 3.1 PITC
def test_pitc_blocks_limits_and_structure():
    # diagonal blocks are those of K_y, entries off them are the Nystrom Q;
    # blocks of one row give FITC, one block of all rows gives K_y
    p = synthetic.make_problem(90, 3, 14, ell=0.9, noise=0.03)
    ell, s2 = oracle.split_theta(p.log_theta, 3, True)
    idx = synthetic.inducing_subset(90, 12, seed=3)
    Pt = oracle.PITC(p.X, ell, s2, p.noise, idx, 25)  # blocks 25, 25, 25, 15
    Ky = _lib_gram(p.X, p.X, ell, s2) + p.noise * np.eye(90)
    KXU = _lib_gram(p.X, p.X[idx], ell, s2)
    Q = KXU @ np.linalg.solve(_lib_gram(p.X[idx], p.X[idx], ell, s2), KXU.T)
    for r0 in (0, 25, 50, 75):
        r1 = min(90, r0 + 25)
        np.testing.assert_allclose(Pt.P[r0:r1, r0:r1], Ky[r0:r1, r0:r1], atol=1e-12)
    np.testing.assert_allclose(Pt.P[:25, 25:], Q[:25, 25:], atol=1e-8)
    np.testing.assert_allclose(Pt.P[75:, :75], Q[75:, :75], atol=1e-8)
    F = oracle.FITC(p.X, ell, s2, p.noise, idx)
    np.testing.assert_allclose(oracle.PITC(p.X, ell, s2, p.noise, idx, 1).P, F.P, atol=1e-12)
    np.testing.assert_allclose(oracle.PITC(p.X, ell, s2, p.noise, idx, 90).P, Ky, atol=1e-12)
    v = synthetic.rng(4).standard_normal(90)
    np.testing.assert_allclose(Pt.P @ Pt.apply(v), v, atol=1e-9 * np.abs(v).max())


# ------------------------------------- Sec. 4 qualitative claims (soft checks)
def test_sec4_low_rank_preconditioners_gain_most_at_long_lengthscales():
    # Sec. 4: Nystrom, FITC and PITC cut iterations most when the lengthscale is
    # long (not at short ones), and block-Jacobi on unordered inputs does not
    # help on a dense K.  A soft check of the paper's claims on synthetic data
    # (isotropic, s2 = 1, noise 1e-4, stop at ||r||^2 < n 1e-10, m = sqrt(n)),
    # not a parity pin: per preconditioner, the best gain over the longer
    # lengthscales 10^0 and 10^0.5 beats the gain at 10^-0.5 and is a real cut.
    n, d = 324, 4
    p = synthetic.make_problem(n, d, 21, dist="standardized", ard=False, ell=1.0)
    m = 18
    idx = synthetic.inducing_subset(n, m, seed=5)
    noise = 1e-4
    gains = {}
    for le in (-0.5, 0.0, 0.5):
        ell = np.full(d, 10.0 ** le)
        Ky = oracle.dense_ky(p.X, ell, 1.0, noise)
        tol = float(np.sqrt(n * 1e-10) / np.linalg.norm(p.y))
        _, it_cg = oracle.pcg_dense(Ky, p.y, lambda r: r, tol=tol)
        pcs = {"nystrom": oracle.Nystrom(p.X, ell, 1.0, noise, idx),
               "fitc": oracle.FITC(p.X, ell, 1.0, noise, idx),
               "pitc": oracle.PITC(p.X, ell, 1.0, noise, idx, m),
               "block_jacobi": oracle.BlockJacobi(p.X, ell, 1.0, noise, m)}
        for k, P in pcs.items():
            _, it = oracle.pcg_dense(Ky, p.y, P.apply, tol=tol)
            gains[(k, le)] = math.log10(max(it, 1) / max(it_cg, 1))
    for k in ("nystrom", "fitc", "pitc"):
        best_long = min(gains[(k, 0.0)], gains[(k, 0.5)])
        assert best_long < gains[(k, -0.5)] and best_long < -0.1, (k, gains)
    assert min(gains[("block_jacobi", 0.0)], gains[("block_jacobi", 0.5)]) > -0.05, gains
