"""Failure detection inside the tensor-core kernels: every mbarrier wait is
bounded.  A wait that runs out records an error, lets the CTA's own bulk
copies land, frees its tensor memory and returns; the call then reports
KPCG_ERR_TIMEOUT and the handle stays usable.

The test makes the wait run out on purpose through the options' test hook:
with wait_stall = 1 the MMA thread first waits on an mbarrier that nothing
ever arrives at, under a 2 ms limit (wait_limit_ns), so the expiry path runs
deterministically.  No GPU fault, trap or unbounded wait is involved.
"""
import numpy as np
import pytest

import oracle
import synthetic

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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("impl", [1, 4, 5, 6])
def test_expired_wait_reports_timeout_and_the_handle_recovers(kpcg, impl):
    p = synthetic.make_problem(3000, 8, 5, dist="normal", ell="loguniform", noise=1e-2)
    V = synthetic.rng(3).standard_normal(p.n)
    Vd = torch.from_numpy(V).to("cuda:0", torch.float32)
    ell, s2 = oracle.split_theta(p.log_theta, p.d, p.ard)
    ref = oracle.kyv(p.X, ell, s2, p.noise, V)
    X = torch.from_numpy(p.X).to("cuda:0")
    with kpcg.Solver(X, p.log_theta, p.noise, ard=True) as s:
        s.set_options(kpcg.default_options(wait_stall=1, wait_limit_ns=2_000_000))
        for _ in range(2):  # twice: the error flag is cleared after each report
            with pytest.raises(kpcg.KpcgError) as e:
                s.matvec_f32(Vd, impl=impl)
            assert e.value.name == "KPCG_ERR_TIMEOUT"
        # the mixed solve built on this kernel reports it too
        opt = kpcg.default_options(precision=kpcg.KPCG_TCX_IR if impl == 4 else kpcg.KPCG_TC_IR,
                                   wait_stall=1, wait_limit_ns=2_000_000, inner_max_iter=4,
                                   max_outer=3)
        s.set_options(opt)
        y = torch.from_numpy(p.y).to("cuda:0")
        with pytest.raises(kpcg.KpcgError) as e:
            s.solve(y, tol=1e-8)
        assert e.value.name == "KPCG_ERR_TIMEOUT"
        # same handle, default options: a normal product, at the parity tolerance
        s.set_options(kpcg.default_options())
        out = s.matvec_f32(Vd, impl=impl).double().cpu().numpy()
        assert _rel(out, ref) <= (5e-6 if impl == 4 else 2e-5)
        torch.cuda.synchronize()


def test_wait_options_are_validated(kpcg):
    p = synthetic.make_problem(200, 3, 1)
    X = torch.from_numpy(p.X).to("cuda:0")
    with kpcg.Solver(X, p.log_theta, p.noise, ard=True) as s:
        for bad in (dict(wait_stall=2), dict(wait_limit_ns=-1)):
            with pytest.raises(kpcg.KpcgError) as e:
                s.set_options(kpcg.default_options(**bad))
            assert e.value.name == "KPCG_ERR_ARG"
