"""The benchmark's roofline arithmetic (host logic, no GPU): the algorithmic
work of one product (K + sigma^2 I) V is that of the distinct entries of the
symmetric K -- one exp2 each, 2d flops for the squared distance and 2c flops
for the contraction with V (row i and, mirrored, column j) -- and `frac` is the
time of the binding resource (MUFU ex2 or tensor cores, at the measured rates)
over the measured time."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = saved
    return mod


RATES = {"ex2_per_s": 10.0e12, "fp32_fma_per_s": 38.6e12, "fp64_fma_per_s": 0.527e12,
         "bf16_tflops": 1934.6}


def test_algorithmic_work_counts_distinct_entries(bench):
    n, d, c = 65536, 8, 1
    w = bench.kv_algorithmic(n, d, c)
    ent = n * (n + 1) / 2
    assert w["distinct_entries"] == ent
    assert w["ex2"] == ent
    assert w["distance_flops"] == 2 * d * ent
    assert w["contraction_flops"] == 2 * n * n * c
    assert w["fp32_slots"] == ent * (2 * d + 2 * c)


def test_frac_is_the_binding_resource_over_the_measured_time(bench):
    n, d, c = 65536, 8, 1
    w = bench.kv_algorithmic(n, d, c)
    t_ex2 = w["ex2"] / RATES["ex2_per_s"]                       # 0.215 ms
    t_ten = (w["distance_flops"] + w["contraction_flops"]) / (RATES["bf16_tflops"] * 1e12)
    assert t_ex2 > t_ten                                         # one column: the MUFU binds
    r = bench.alu_roofline("k", n, d, c, ms=2 * t_ex2 * 1e3, rates=RATES)
    assert r["pipe"] == "mufu_ex2" and r["unit"] == "Tex2/s"
    assert r["frac"] == pytest.approx(0.5)
    assert r["frac_evaluated"] == pytest.approx(1.0)             # all n^2 entries
    assert r["achieved"] == pytest.approx(w["ex2"] / (2 * t_ex2) / 1e12)
    assert r["peak"] == pytest.approx(RATES["ex2_per_s"] / 1e12)


def test_many_columns_make_the_tensor_cores_bind(bench):
    # the augmented derivative product's width (323 columns) is tensor-bound
    n, d, c = 45730, 9, 323
    w = bench.kv_algorithmic(n, d, c)
    r = bench.roofline_from_work("k", w, 10.0, RATES)
    t_ten = (w["distance_flops"] + w["contraction_flops"]) / (RATES["bf16_tflops"] * 1e12)
    assert r["pipe"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(t_ten / 10e-3)


def test_fp64_certification_counts_its_pipe(bench):
    n, d, c = 65536, 8, 1
    w = bench.kv_algorithmic(n, d, c)
    ms = 119.5
    r = bench.alu_roofline("k", n, d, c, ms, RATES, fp64=True)
    assert r["pipe"] == "fp64"
    assert r["frac"] == pytest.approx((w["fp32_slots"] + w["ex2"]) / RATES["fp64_fma_per_s"]
                                      / (ms / 1e3))


def test_traffic_is_known_only_for_kernels_measured_since_their_last_change(bench):
    # DRAM bytes per launch scale with n (operands read once) ...
    t = bench.known_traffic("kv_tcds_kernel (double-float) (outer directions)", 65536)
    assert t == pytest.approx(4 * bench.known_traffic("kv_tcds_kernel", 16384))
    # ... and kernels changed since their capture carry none
    assert bench.known_traffic("kv_f64_sym_kernel (certification)", 65536) is None
    assert bench.known_traffic("kv_tcs_kernel", 65536) is None
