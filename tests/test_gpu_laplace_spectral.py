"""GPU parity of the random-feature preconditioner (Sec. 3.2) and of the probit
Laplace mode (Sec. 2.2, Appendix B) against the FP64 oracle.

Inputs are seeded and synthetic (``synthetic``): the random-feature draws are
passed to both sides, the labels come from a smooth signal with flipped
labels.  Tolerances:
  * spectral apply: 1e-9 relative (FP64 on both sides; the GPU stores Phi as
    exact FP32 pairs and applies the inversion lemma, the oracle factors P).
  * spectral solves: the iteration count of textbook PCG with the oracle's
    preconditioner within max(2, 5%), the solution within 1e-7 of Cholesky.
  * Laplace: the same Newton step count (+-1), f^ and a within 1e-7 relative,
    Psi within 1e-10 relative: each B-solve is certified at 1e-10, and the
    Newton map damps the solve error at the mode.
"""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def kpcg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_06693_gb300 as k
    from paper_1602_06693_gb300 import build
    build.build()
    return k


def _cm(a):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).to(DEV)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(DEV).t()


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _solver(kpcg, p, precision=None, **kw):
    opt = kpcg.default_options(**kw)
    if precision is not None:
        opt.precision = precision
    return kpcg.Solver(torch.from_numpy(p.X).to(DEV), p.log_theta, p.noise, ard=p.ard,
                       options=opt)


# ------------------------------------------------------------ spectral (Sec. 3.2)
@pytest.mark.parametrize("n,d,m,ard", [(900, 5, 60, True), (1500, 3, 200, False),
                                       (700, 24, 40, True)])
def test_spectral_apply_matches_oracle(kpcg, n, d, m, ard):
    p = synthetic.make_problem(n, d, seed=n + d, ard=ard, ell=1.2, noise=0.05)
    ell, s2 = oracle.split_theta(p.log_theta, d, ard)
    om = synthetic.spectral_draws(m, d, seed=3)
    S = oracle.Spectral(p.X, ell, s2, p.noise, om)
    R = synthetic.rng(4).standard_normal((n, 3))
    with _solver(kpcg, p, precision=kpcg.KPCG_FP64) as s:
        s.precond_spectral(om)
        Z = _np(s.precond_apply(_cm(R)))
    for k in range(3):
        assert _rel(Z[:, k], S.apply(R[:, k])) <= 1e-9, k


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_spectral_solve_matches_oracle(kpcg, precision):
    p = synthetic.make_problem(1200, 4, seed=21, ell="loguniform", noise=0.02)
    ell, s2 = oracle.split_theta(p.log_theta, 4, True)
    om = synthetic.spectral_draws(100, 4, seed=5)
    S = oracle.Spectral(p.X, ell, s2, p.noise, om)
    prec = kpcg.KPCG_FP64 if precision == "fp64" else kpcg.KPCG_DF64
    with _solver(kpcg, p, precision=prec) as s:
        s.precond_spectral(om)
        x, it, info, st = s.solve(_cm(p.y), tol=1e-10)
    assert st == 0
    Ky = oracle.dense_ky(p.X, ell, s2, p.noise)
    ref_tol = 1e-10 if precision == "fp64" else 0.5e-10
    _, it_ref = oracle.pcg_dense(Ky, p.y, S.apply, tol=ref_tol)
    _, it_none = oracle.pcg_dense(Ky, p.y, lambda r: r, tol=ref_tol)
    assert _rel(_np(x), oracle.dense_solve(p.X, ell, s2, p.noise, p.y[:, None])[:, 0]) <= 1e-7
    assert abs(int(it[0]) - it_ref) <= max(2, 0.05 * it_ref), (int(it[0]), it_ref)
    assert it_ref < it_none  # the features do precondition


def test_spectral_in_the_mixed_solver_and_after_set_theta(kpcg):
    # the FP32 inner apply goes through the batched Nystrom kernels (K_UU = I);
    # after set_theta the same draws are rescaled by the new lengthscales
    p = synthetic.make_problem(2500, 6, seed=23, ell=1.0, noise=0.01)
    om = synthetic.spectral_draws(150, 6, seed=6)
    with _solver(kpcg, p, precision=kpcg.KPCG_TC_IR, inner_shift=0.25, inner_tol=0.1) as s:
        s.precond_spectral(om)
        x, it, info, st = s.solve(_cm(p.y), tol=1e-8)
        assert st == 0 and info.max_rel_res <= 1e-8
        lt2 = p.log_theta + np.log(1.3)
        s.set_theta(lt2, p.noise)
        s.set_options(kpcg.default_options(precision=kpcg.KPCG_FP64))
        R = synthetic.rng(7).standard_normal((2500, 2))
        Z = _np(s.precond_apply(_cm(R)))
    ell2, s22 = oracle.split_theta(lt2, 6, True)
    S2 = oracle.Spectral(p.X, ell2, s22, p.noise, om)
    for k in range(2):
        assert _rel(Z[:, k], S2.apply(R[:, k])) <= 1e-9


def test_spectral_argument_errors(kpcg):
    p = synthetic.make_problem(300, 3, seed=2)
    with _solver(kpcg, p) as s:
        with pytest.raises(kpcg.KpcgError):
            s.precond(kpcg.KPCG_PREC_SPECTRAL, 10, np.arange(10))
        with pytest.raises(kpcg.KpcgError):
            s.precond_spectral(np.zeros((0, 3)))
        bad = synthetic.spectral_draws(4, 3, seed=1)
        bad[2, 1] = np.nan
        with pytest.raises(kpcg.KpcgError):
            s.precond_spectral(bad)


# ----------------------------------------------- Laplace (Sec. 2.2, Appendix B)
def _laplace_parity(kpcg, p, m, precision=None):
    ell, s2 = oracle.split_theta(p.log_theta, p.d, True)
    ref = oracle.laplace_probit(p.X, ell, s2, p.y, tol=1e-12)
    prec = kpcg.KPCG_DF64 if precision is None else precision
    with _solver(kpcg, p, precision=prec) as s:
        if m:
            s.precond(kpcg.KPCG_PREC_NYSTROM, m, synthetic.inducing_subset(p.n, m, seed=11))
        f, a, info, st = s.laplace(_cm(p.y), newton_tol=1e-12, cg_tol=1e-10)
    assert st == 0
    assert abs(info.newton_steps - ref["steps"]) <= 1, (info.newton_steps, ref["steps"])
    assert _rel(_np(f), ref["f"]) <= 1e-7
    assert _rel(_np(a), ref["a"]) <= 1e-7
    assert abs(info.psi - ref["psi"]) <= 1e-10 * abs(ref["psi"])
    assert info.max_rel_res <= 1e-10
    return info


def test_laplace_matches_oracle_with_and_without_preconditioner(kpcg):
    p = synthetic.classification_problem(1500, 6, seed=31, s2=4.0, ell=1.5)
    plain = _laplace_parity(kpcg, p, 0)
    nys = _laplace_parity(kpcg, p, 120)
    # the Nystrom form of B needs fewer CG iterations over the Newton loop
    assert nys.cg_iters_total < plain.cg_iters_total, (nys.cg_iters_total,
                                                        plain.cg_iters_total)


@pytest.mark.parametrize("mode", ["tc_ir", "fp32_ir"])
@pytest.mark.parametrize("m", [0, 120])
def test_laplace_mixed_precision_b_solves_match_oracle(kpcg, mode, m):
    # the B-solves as flexible CG around FP32 / tensor-core inner solves: same
    # mode, same Newton steps, certified residuals at 1e-10
    p = synthetic.classification_problem(1500, 6, seed=31, s2=4.0, ell=1.5)
    prec = kpcg.KPCG_TC_IR if mode == "tc_ir" else kpcg.KPCG_FP32_IR
    _laplace_parity(kpcg, p, m, precision=prec)


def test_laplace_credit_shape_matches_oracle(kpcg):
    # n = 1000, d = 24: the padded dimension 32 takes the row-split kernels
    p = synthetic.credit_shape(seed=2)
    _laplace_parity(kpcg, p, 64)


def test_laplace_eeg_shape_is_stationary(kpcg):
    # full EEG shape (n = 14979, d = 14).  The mode condition grad Psi =
    # g(f^) - K^{-1} f^ = 0 reads a = g(f^) for f^ = K a: the product on sampled
    # rows (each row of K from the oracle) and a = g(f^) on every row.  (The
    # form f^ = K g(f^) multiplies the B-solve error by |K| ~ 2e4 here.)
    p = synthetic.eeg_shape(seed=0)
    ell, s2 = oracle.split_theta(p.log_theta, 14, True)
    with _solver(kpcg, p, precision=kpcg.KPCG_DF64) as s:
        s.precond(kpcg.KPCG_PREC_NYSTROM, 512, synthetic.inducing_subset(p.n, 512, seed=12))
        f, a, info, st = s.laplace(_cm(p.y), newton_tol=1e-12, cg_tol=1e-10)
    assert st == 0 and 3 <= info.newton_steps <= 15
    f, a = _np(f), _np(a)
    _, g, _ = oracle.probit_terms(p.y, f)
    assert _rel(a, g) <= 1e-6, _rel(a, g)
    rows = np.arange(0, p.n, 373)
    Ka = oracle.gram(p.X[rows], p.X, ell, s2) @ a
    assert np.abs(Ka - f[rows]).max() <= 1e-8 * np.abs(f).max()
    assert np.mean(np.sign(f) == p.y) > 0.85


def test_laplace_argument_errors(kpcg):
    p = synthetic.classification_problem(400, 3, seed=3)
    with _solver(kpcg, p) as s:
        y = p.y.copy()
        y[5] = 0.5
        with pytest.raises(kpcg.KpcgError):
            s.laplace(_cm(y))
        s.precond(kpcg.KPCG_PREC_BLOCK_JACOBI, 64)
        with pytest.raises(kpcg.KpcgError):
            s.laplace(_cm(p.y))
        s.precond(kpcg.KPCG_PREC_NONE)
        f, a, info, st = s.laplace(_cm(p.y), max_newton=1)
        assert st == 6 and info.newton_steps == 1  # stopped before the test was met


# ---------------------------------------- probit predictions (Sec. 2.2, App. B)
@pytest.mark.parametrize("m,mode", [(0, "df64"), (90, "df64"), (90, "tc_ir")])
def test_laplace_predictions_match_oracle(kpcg, m, mode):
    # mean from a (FP64 on both sides), variance through one B-solve per test
    # point (blocks of 16; 37 points leave a ragged block of 5), probability
    p = synthetic.classification_problem(1200, 5, seed=41, s2=3.0, ell=1.4)
    ell, s2 = oracle.split_theta(p.log_theta, 5, True)
    ref = oracle.laplace_probit(p.X, ell, s2, p.y, tol=1e-12)
    Xs = synthetic.rng(42).standard_normal((37, 5)).astype(np.float32)
    Xs[3] = p.X[10]  # a training input
    Xs[4] = 40.0     # far from the data: the prior
    mr, vr, pr = oracle.laplace_predict(p.X, ell, s2, p.y, ref["f"], ref["a"], Xs)
    prec = kpcg.KPCG_TC_IR if mode == "tc_ir" else kpcg.KPCG_DF64
    with _solver(kpcg, p, precision=prec) as s:
        if m:
            s.precond(kpcg.KPCG_PREC_NYSTROM, m, synthetic.inducing_subset(p.n, m, seed=13))
        y = _cm(p.y)
        f, a, info, st = s.laplace(y, newton_tol=1e-12, cg_tol=1e-10)
        assert st == 0
        mean, var, prob, pinfo = s.laplace_predict(y, f, a, torch.from_numpy(Xs).to(DEV))
    mean, var, prob = _np(mean), _np(var), _np(prob)
    # the GPU's own mode agrees with the oracle's to ~1e-7 (the B-solves are
    # certified at 1e-10); predictions inherit that, with one more B-solve each
    assert np.abs(mean - mr).max() <= 1e-6 * max(1.0, np.abs(mr).max())
    assert np.abs(var - vr).max() <= 1e-6 * s2
    assert np.abs(prob - pr).max() <= 1e-6
    assert abs(mean[4]) < 1e-12 and var[4] == pytest.approx(s2, rel=1e-12)
    assert pinfo.max_rel_res <= 1e-10 and pinfo.cg_iters_total > 0


def test_laplace_predict_mean_only_and_empty(kpcg):
    p = synthetic.classification_problem(500, 3, seed=43)
    with _solver(kpcg, p, precision=kpcg.KPCG_DF64) as s:
        y = _cm(p.y)
        f, a, info, st = s.laplace(y)
        Xs = torch.from_numpy(synthetic.rng(44).standard_normal((3, 3)).astype(np.float32)).to(DEV)
        mean, var, prob, pinfo = s.laplace_predict(y, f, a, Xs, var=False, prob=False)
        assert var is None and prob is None and pinfo.cg_iters_total == 0
        mean0, _, _, _ = s.laplace_predict(y, f, a, Xs[:0])
        assert mean0.numel() == 0
    ell, s2 = oracle.split_theta(p.log_theta, 3, True)
    ref = oracle.gram(_np(Xs), p.X, ell, s2) @ _np(a)
    assert _rel(_np(mean), ref) <= 1e-12


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("n", [1, 2, 129])
def test_laplace_small_and_ragged_sizes(kpcg, n):
    # n = 1 (one label, the scalar Newton of the one-point closed form), n = 2,
    # and one row past a 128-row tile; predictions at 1 and 16 test points
    p = synthetic.classification_problem(max(n, 2), 3, seed=50 + n, s2=2.0, ell=1.0)
    X, y = p.X[:n], p.y[:n]
    ell, s2 = oracle.split_theta(p.log_theta, 3, True)
    ref = oracle.laplace_probit(X, ell, s2, y, tol=1e-12)
    opt = kpcg.default_options(precision=kpcg.KPCG_DF64)
    with kpcg.Solver(torch.from_numpy(np.ascontiguousarray(X)).to(DEV), p.log_theta, 1.0,
                     ard=True, options=opt) as s:
        yd = _cm(y)
        f, a, info, st = s.laplace(yd, newton_tol=1e-12, cg_tol=1e-10)
        assert st == 0 and abs(info.newton_steps - ref["steps"]) <= 1
        assert _rel(_np(f), ref["f"]) <= 1e-7
        for ns in (1, 16):
            Xs = synthetic.rng(60 + ns).standard_normal((ns, 3)).astype(np.float32)
            mean, var, prob, _ = s.laplace_predict(yd, f, a, torch.from_numpy(Xs).to(DEV))
            mr, vr, pr = oracle.laplace_predict(X, ell, s2, y, ref["f"], ref["a"], Xs)
            assert np.abs(_np(var) - vr).max() <= 1e-6 * s2
            assert np.abs(_np(prob) - pr).max() <= 1e-6


def test_spectral_single_frequency(kpcg):
    # m = 1: Phi has two columns (one cosine, one sine)
    p = synthetic.make_problem(300, 2, seed=61, ell=0.8, noise=0.1)
    ell, s2 = oracle.split_theta(p.log_theta, 2, True)
    om = synthetic.spectral_draws(1, 2, seed=62)
    S = oracle.Spectral(p.X, ell, s2, p.noise, om)
    R = synthetic.rng(63).standard_normal((300, 2))
    with _solver(kpcg, p, precision=kpcg.KPCG_FP64) as s:
        s.precond_spectral(om)
        Z = _np(s.precond_apply(_cm(R)))
    for k in range(2):
        assert _rel(Z[:, k], S.apply(R[:, k])) <= 1e-9


# -------------------------------------------------------------- PITC (Sec. 3.1)
@pytest.mark.parametrize("n,d,m,b", [(1000, 4, 50, 64), (700, 6, 30, 1), (513, 3, 40, 513)])
def test_pitc_apply_matches_oracle(kpcg, n, d, m, b):
    # 15 blocks of 64 and a ragged one of 40; b = 1 (FITC); one block (K_y itself)
    p = synthetic.make_problem(n, d, seed=n + b, ell=1.1, noise=0.03)
    ell, s2 = oracle.split_theta(p.log_theta, d, True)
    idx = synthetic.inducing_subset(n, m, seed=8)
    Pt = oracle.PITC(p.X, ell, s2, p.noise, idx, b)
    R = synthetic.rng(9).standard_normal((n, 3))
    with _solver(kpcg, p, precision=kpcg.KPCG_FP64) as s:
        s.precond_pitc(m, idx, b)
        Z = _np(s.precond_apply(_cm(R)))
    for k in range(3):
        assert _rel(Z[:, k], Pt.apply(R[:, k])) <= 1e-9, k


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_pitc_solve_matches_oracle(kpcg, precision):
    p = synthetic.make_problem(1100, 5, seed=71, ell="loguniform", noise=0.01)
    ell, s2 = oracle.split_theta(p.log_theta, 5, True)
    idx = synthetic.inducing_subset(1100, 60, seed=10)
    Pt = oracle.PITC(p.X, ell, s2, p.noise, idx, 100)
    prec = kpcg.KPCG_FP64 if precision == "fp64" else kpcg.KPCG_DF64
    with _solver(kpcg, p, precision=prec) as s:
        s.precond_pitc(60, idx, 100)
        x, it, info, st = s.solve(_cm(p.y), tol=1e-10)
    assert st == 0
    Ky = oracle.dense_ky(p.X, ell, s2, p.noise)
    ref_tol = 1e-10 if precision == "fp64" else 0.5e-10
    _, it_ref = oracle.pcg_dense(Ky, p.y, Pt.apply, tol=ref_tol)
    assert _rel(_np(x), oracle.dense_solve(p.X, ell, s2, p.noise, p.y[:, None])[:, 0]) <= 1e-7
    assert abs(int(it[0]) - it_ref) <= max(2, 0.05 * it_ref), (int(it[0]), it_ref)


def test_pitc_in_the_mixed_solver_and_errors(kpcg):
    p = synthetic.make_problem(2000, 6, seed=73, noise=0.01)
    idx = synthetic.inducing_subset(2000, 100, seed=11)
    with _solver(kpcg, p, precision=kpcg.KPCG_TC_IR, inner_shift=0.25, inner_tol=0.1) as s:
        s.precond_pitc(100, idx, 45)
        x, it, info, st = s.solve(_cm(p.y), tol=1e-8)
        assert st == 0 and info.max_rel_res <= 1e-8
        with pytest.raises(kpcg.KpcgError):
            s.precond(kpcg.KPCG_PREC_PITC, 100, idx)
        with pytest.raises(kpcg.KpcgError):
            s.precond_pitc(100, idx, 0)
