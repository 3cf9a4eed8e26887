"""GPU tests of the learned warm start: the network's kernels against the FP64
oracle (oracle/mlp.py), the basis fit and expansion against a dense FP64
least-squares solution, and the gain of the trained network over cold starts
along a short hyperparameter trajectory."""
import math

import numpy as np
import pytest

import oracle
import synthetic
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kpcg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_06693_gb300 as k
    from paper_1602_06693_gb300 import build
    build.build()
    return k


def _case(n_in=12, h=64, n_out=96, B=40, seed=3):
    P = synthetic.mlp_init(seed, n_in, h, h, n_out)
    X = synthetic.rng(seed + 1).standard_normal((B, n_in))
    T = synthetic.rng(seed + 2).standard_normal((B, n_out))
    # parameters and data as the GPU sees them (float32), widened for the oracle
    P32 = {k: v.astype(np.float32).astype(np.float64) for k, v in P.items()}
    return P, P32, X.astype(np.float32), T.astype(np.float32)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_mlp_forward_and_gradient_match_oracle(kpcg):
    # FP32 kernels vs the FP64 reference: forward within 1e-5, gradients within
    # 1e-4 of their largest entry (FP32 sums over <= 64 terms per product).
    P, P32, X, T = _case()
    net = kpcg.MLP(P)
    out = net.forward(_t(X)).cpu().numpy()
    ref, _ = omlp.forward(P32, X.astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    g, loss = net.grad(_t(X), _t(T))
    gref = omlp.backward(P32, X.astype(np.float64), T.astype(np.float64))
    for k in omlp.NAMES:
        np.testing.assert_allclose(g[k], gref[k], rtol=1e-4, atol=1e-4 * np.abs(gref[k]).max())
    assert loss == pytest.approx(omlp.loss(P32, X, T), rel=1e-5)


def test_mlp_adam_steps_match_oracle(kpcg):
    P, P32, X, T = _case(seed=5)
    net = kpcg.MLP(P)
    net.train(_t(X), _t(T), epochs=3, lr=1e-2)
    got = net.params()
    ref = {k: v.copy() for k, v in P32.items()}
    state = {}
    for _ in range(3):
        ref = omlp.adam_step(ref, omlp.backward(ref, X.astype(np.float64), T.astype(np.float64)),
                             state, lr=1e-2)
    for k in omlp.NAMES:
        np.testing.assert_allclose(got[k], ref[k], rtol=2e-4, atol=2e-4 * np.abs(ref[k]).max())


def test_mlp_bf16_inference_close_to_fp32(kpcg):
    # BF16 weights and inputs (8-bit mantissa), FP32 accumulation: ~1e-2 relative.
    P, _, X, _ = _case(seed=7)
    net = kpcg.MLP(P)
    a = net.forward(_t(X)).cpu().numpy()
    b = net.forward(_t(X), bf16=True).cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(a) <= 2e-2


def test_warm_basis_fit_and_expand_match_least_squares(kpcg):
    p = synthetic.make_problem(1500, 5, 3, ell=1.2, noise=0.05)
    idx = synthetic.inducing_subset(1500, 60, seed=2)
    ridge = 1e-6
    a = synthetic.rng(4).standard_normal(1500)
    with kpcg.Solver(torch.from_numpy(p.X).cuda(), p.log_theta, p.noise) as s:
        s.warm_basis(idx, ridge)
        c = s.warm_fit(torch.from_numpy(a).cuda())
        x0 = s.warm_expand(c).cpu().numpy()
        c = c.cpu().numpy()
    ell, s2 = oracle.split_theta(p.log_theta, 5, True)
    KXZ = oracle.gram(p.X, p.X[idx], ell, s2)
    KZZ = KXZ[idx]
    cref = np.linalg.solve(KXZ.T @ KXZ + ridge * KZZ, KXZ.T @ a)

    def objective(v):  # the ridge least-squares functional the fit minimises
        r = a - KXZ @ v
        return r @ r + ridge * v @ KZZ @ v

    # c itself can be ill-determined (M = K_ZX K_XZ + ridge K_ZZ is badly
    # conditioned), so compare what is unique: the minimum and the fitted vector
    assert objective(c) <= objective(cref) * (1 + 1e-9)
    fit, fref = KXZ @ c, KXZ @ cref
    assert np.linalg.norm(fit - fref) / np.linalg.norm(fref) <= 1e-6
    np.testing.assert_allclose(x0, fit, rtol=1e-10, atol=1e-10 * np.abs(x0).max())


def test_trained_network_cuts_pcg_iterations(kpcg):
    # A short Adam trajectory on (log l_1..d, log s^2, log noise): the first 12
    # steps train the network, the next 12 start PCG from its prediction.
    from paper_1602_06693_gb300.warmstart import Trajectory
    n, d = 2048, 6
    p = synthetic.make_problem(n, d, 11, dist="normal", ell=1.0, noise=0.1)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    opt = kpcg.default_options(precision=kpcg.KPCG_FP64, max_iter=2000)
    s = kpcg.Solver(X, p.log_theta, p.noise, options=opt)
    basis = synthetic.inducing_subset(n, 256, seed=5)
    pidx = synthetic.inducing_subset(n, 128, seed=6)
    probes = lambda k: torch.from_numpy(synthetic.rademacher(n, 4, 1000 + k)).cuda()
    params = synthetic.mlp_init(9, d + 2, 128, 128, 256)
    tr = Trajectory(s, y, basis, pidx, probes, lr=0.05, n_train=12, mlp_params=params,
                    epochs=1500, mlp_lr=2e-3, tol=1e-8, compare=True)
    z0 = np.concatenate([p.log_theta, [math.log(p.noise)]])
    recs = tr.run(z0, 24)
    assert all(r.rel_res <= 1e-8 for r in recs)
    warm = [r for r in recs if r.warm]
    assert len(warm) == 12
    w = np.array([r.iters for r in warm])
    c = np.array([r.cold_iters for r in warm])
    print("same theta: cold iterations", c.tolist(), "warm iterations", w.tolist())
    # paired at the same theta, the warm starts must save iterations at every step
    assert np.all(w < c), (c, w)
    assert w.sum() <= 0.85 * c.sum(), (c, w)
    s.close()
