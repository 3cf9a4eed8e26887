"""kpcg_matvec_f64_noalloc: the FP64 kernel product for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or they
must avoid cudaMalloc's device synchronisation).  Its scratch is a static
device array inside the library.  Checked through the C ABI against the
handle-based kpcg_matvec_f64 (impl 0) on two calls in a row, at the FP64
tolerance of the parity tests; this file is collected last on purpose.
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


def _cm(a):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).to("cuda:0")
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda:0").t()


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_handle_product_on_two_calls(kpcg):
    cases = [(synthetic.make_problem(3000, 8, 1, dist="uniform", ell="loguniform", noise=1e-4), 3),
             (synthetic.make_problem(1337, 5, 2, ard=False, ell=0.8, noise=0.02), 1)]
    for p, c in cases:  # two calls in a row share (and overwrite) the static scratch
        X = torch.from_numpy(p.X).to("cuda:0")
        V = _cm(synthetic.rng(4).standard_normal((p.n, c)))
        with kpcg.Solver(X, p.log_theta, p.noise, ard=p.ard) as s:
            ref = s.matvec_f64(V, impl=0)
        got = kpcg.matvec_f64_noalloc(X, p.log_theta, p.noise, V, ard=p.ard)
        torch.cuda.synchronize()
        assert got.shape == ref.shape
        assert _rel(got, ref) <= 1e-12


def test_noalloc_matches_oracle_on_a_side_stream(kpcg):
    # More than four columns (two passes of the column-block loop over the
    # shared scratch), padded dimensions 12 and 16, an explicit non-default
    # stream; compared with the FP64 oracle directly and with impl 0.
    side = torch.cuda.Stream()
    for n, d, c in ((2100, 12, 6), (1500, 16, 5)):
        p = synthetic.make_problem(n, d, 10 + d, dist="normal", ell="loguniform", noise=1e-3)
        Vn = synthetic.rng(11).standard_normal((n, c))
        ell, s2 = oracle.split_theta(p.log_theta, d, p.ard)
        ref = oracle.kyv(p.X, ell, s2, p.noise, Vn)
        X = torch.from_numpy(p.X).to("cuda:0")
        V = _cm(Vn)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            got = kpcg.matvec_f64_noalloc(X, p.log_theta, p.noise, V, ard=p.ard, stream=side)
        side.synchronize()
        got_np = got.cpu().numpy()
        assert np.linalg.norm(got_np - ref) / np.linalg.norm(ref) <= 1e-12
        with kpcg.Solver(X, p.log_theta, p.noise, ard=p.ard) as s:
            h = s.matvec_f64(V, impl=0)
        assert _rel(got, h) <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch(kpcg):
    n, d = 1 << 20, 8  # needs more than the 16 MiB static scratch
    X = torch.zeros((n, d), dtype=torch.float32, device="cuda:0")
    V = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(kpcg.KpcgError) as e:
        kpcg.matvec_f64_noalloc(X, np.zeros(d + 1), 0.1, V)
    assert e.value.name == "KPCG_ERR_ARG" and "scratch" in str(e.value)
