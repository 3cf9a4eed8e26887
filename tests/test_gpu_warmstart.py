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


def test_mlp_bf16_inference_matches_oracle(kpcg):
    # BF16 weights and inputs (8 significant bits, relative rounding <= 2^-9 per
    # value), FP32 accumulation.  Against the FP64 forward of the same float32
    # parameters: the output error is a sum of such roundings through three
    # layers (tanh is 1-Lipschitz), bounded here by 2e-2 of the output norm and
    # 5e-2 of the largest output per entry; and the BF16 forward stays within
    # the same bound of the GPU's own FP32 forward.
    P, P32, X, _ = _case(seed=7)
    net = kpcg.MLP(P)
    b = net.forward(_t(X), bf16=True).cpu().numpy()
    ref, _ = omlp.forward(P32, X.astype(np.float64))
    assert np.linalg.norm(b - ref) / np.linalg.norm(ref) <= 2e-2
    assert np.abs(b - ref).max() <= 5e-2 * np.abs(ref).max()
    a = net.forward(_t(X)).cpu().numpy()
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


def _trajectory(kpcg, basis, n_train=12, steps=24):
    from paper_1602_06693_gb300.warmstart import Trajectory
    n, d = 2048, 6
    p = synthetic.make_problem(n, d, 11, dist="normal", ell=1.0, noise=0.1)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    opt = kpcg.default_options(precision=kpcg.KPCG_FP64, max_iter=2000)
    s = kpcg.Solver(X, p.log_theta, p.noise, options=opt)
    pidx = synthetic.inducing_subset(n, 128, seed=6)
    probes = lambda k: torch.from_numpy(synthetic.rademacher(n, 4, 1000 + k)).cuda()
    q_out = 4 if basis == "snapshots" else 256
    params = synthetic.mlp_init(9, d + 2, 128, 128, q_out)
    tr = Trajectory(s, y, pidx, probes, basis=basis, q=4,
                    basis_idx=synthetic.inducing_subset(n, 256, seed=5), lr=0.05,
                    n_train=n_train, mlp_params=params, epochs=1500, mlp_lr=2e-3, tol=1e-8,
                    compare=True)
    z0 = np.concatenate([p.log_theta, [math.log(p.noise)]])
    recs = tr.run(z0, steps)
    s.close()
    assert all(r.rel_res <= 1e-8 for r in recs)
    warm = [r for r in recs if r.warm]
    assert len(warm) == steps - n_train
    w = np.array([r.iters for r in warm])
    c = np.array([r.cold_iters for r in warm])
    print(basis, "same theta: cold iterations", c.tolist(), "warm iterations", w.tolist())
    return c, w


def test_trained_network_cuts_pcg_iterations(kpcg):
    # Adam on (log l_1..d, log s^2, log noise); steps 4..11 give training pairs
    # (coefficients of alpha_k on the 4 solutions before it), steps 12..23
    # start PCG from the network's prediction.  Paired with a cold start at
    # the same theta, the network must save iterations at every step and a
    # fifth of them overall (exact least-squares coefficients save about a
    # third on this trajectory).
    c, w = _trajectory(kpcg, "snapshots")
    assert np.all(w < c), (c, w)
    assert w.sum() <= 0.8 * c.sum(), (c, w)


def test_kernel_basis_warm_start_is_safe(kpcg):
    # On the smooth basis K(X, Z) even exact coefficients save ~3% here; the
    # learned start must not cost more than a few iterations over cold.
    c, w = _trajectory(kpcg, "kernel")
    assert np.all(w <= c + 4), (c, w)


def test_snapshot_fit_and_expand_match_least_squares(kpcg):
    n = 900
    p = synthetic.make_problem(n, 4, 5, noise=0.1)
    S = synthetic.rng(8).standard_normal((n, 5))
    a = S[:, :3] @ np.array([0.5, -1.0, 2.0]) + 1e-3 * synthetic.rng(9).standard_normal(n)
    with kpcg.Solver(torch.from_numpy(p.X).cuda(), p.log_theta, p.noise) as s:
        s.warm_snapshots(3, 1e-12)
        for j in range(5):  # the ring keeps the last three: S[:, 2], S[:, 3], S[:, 4]
            s.warm_push(torch.from_numpy(S[:, j].copy()).cuda())
        c = s.warm_fit(torch.from_numpy(a).cuda())
        x0 = s.warm_expand(c).cpu().numpy()
        c = c.cpu().numpy()
    B = S[:, [4, 3, 2]]  # newest first
    cref = np.linalg.lstsq(B, a, rcond=None)[0]
    np.testing.assert_allclose(c, cref, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(x0, B @ c, rtol=1e-12, atol=1e-12 * np.abs(x0).max())
