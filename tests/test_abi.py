"""CPU-side checks of the C ABI boundary: the library builds for sm_103a,
loads, and exports every entry point that include/kpcg.h declares.  No
compute call is made (there is no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kpcg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1602_06693_gb300 import build
    build.build()
    return build.LIB


def test_header_declares_core_calls():
    names = _declared()
    for core in ("kpcg_create", "kpcg_precond", "kpcg_solve", "kpcg_grad", "kpcg_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(built):
    import ctypes
    L = ctypes.CDLL(built)
    missing = [s for s in _declared() if not hasattr(L, s)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol(built):
    import paper_1602_06693_gb300 as kpcg
    from paper_1602_06693_gb300 import binding
    assert sorted(binding.SYMBOLS) == _declared()
    assert sorted(kpcg.exported_symbols()) == _declared()


def test_default_options_and_status_strings(built):
    import paper_1602_06693_gb300 as kpcg
    o = kpcg.default_options()
    assert o.max_iter == 100000 and o.tol_mode == 0 and 0 < o.inner_tol < 1
    L = kpcg.lib()
    assert L.kpcg_status_string(0) == b"KPCG_OK"
    assert L.kpcg_status_string(6) == b"KPCG_ERR_NO_CONVERGENCE"


def test_create_rejects_host_pointer_without_gpu(built):
    # A host pointer is refused with KPCG_ERR_ARG (or a CUDA error when no
    # driver is present); the library never falls back to the CPU.
    import ctypes
    import numpy as np
    import paper_1602_06693_gb300 as kpcg
    L = kpcg.lib()
    X = np.zeros((4, 2), dtype=np.float32)
    lt = np.zeros(3)
    h = ctypes.c_void_p()
    st = L.kpcg_create(ctypes.c_void_p(X.ctypes.data), 4, 2,
                       lt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, 0.1, None, None,
                       ctypes.byref(h))
    assert st != 0 and not h.value
    assert L.kpcg_last_error(None)


def test_noalloc_rejects_host_pointers_without_gpu(built):
    # The allocation-free product validates X, V and O before any launch: host
    # memory is refused with KPCG_ERR_ARG (here no driver or device exists).
    import ctypes
    import numpy as np
    import paper_1602_06693_gb300 as kpcg
    L = kpcg.lib()
    X = np.zeros((4, 2), dtype=np.float32)
    V = np.zeros(4)
    O = np.zeros(4)
    lt = np.zeros(3)
    st = L.kpcg_matvec_f64_noalloc(ctypes.c_void_p(X.ctypes.data), 4, 2,
                                   lt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, 0.1,
                                   ctypes.c_void_p(V.ctypes.data), 4, 1,
                                   ctypes.c_void_p(O.ctypes.data), 4, None)
    assert st == 1, st  # KPCG_ERR_ARG
    assert b"pointer" in L.kpcg_last_error(None)


def test_oracle_and_library_share_no_code():
    # The oracle is plain C in oracle/, the CUDA path lives in the package:
    # neither includes or imports the other.
    csrc = os.path.join(ROOT, "paper_1602_06693_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".cu", ".cuh", ".py", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower() or f == "__init__.py", f
    otxt = open(os.path.join(ROOT, "oracle", "kpcg_oracle.c")).read()
    assert "kpcg.h" not in otxt and "csrc" not in otxt


def test_null_handle_is_an_argument_error(built):
    # every handle call checks its handle before touching the device
    import ctypes
    import paper_1602_06693_gb300 as kpcg
    L = kpcg.lib()
    nul = ctypes.c_void_p()
    assert L.kpcg_precond_spectral(nul, 4, None) == 1
    assert L.kpcg_precond_pitc(nul, 4, None, 8) == 1
    assert L.kpcg_laplace(nul, None, 1e-12, 10, 1e-10, None, None, None) == 1
    assert L.kpcg_laplace_predict(nul, None, None, None, None, 3, None, None, None, 1e-10,
                                  None) == 1
    assert kpcg.KPCG_PREC_SPECTRAL == 4 and kpcg.KPCG_PREC_PITC == 5
    assert ctypes.sizeof(kpcg.LaplaceInfo) == 4 + 4 + 8 * 4 + 4 + 4


def test_classification_and_spectral_inputs():
    # seeded, +-1 labels of both signs, standardized columns, standard-normal draws
    import numpy as np
    import synthetic
    p = synthetic.classification_problem(500, 6, seed=3)
    assert p.X.dtype == np.float32 and p.X.shape == (500, 6) and p.ard
    assert set(np.unique(p.y)) == {-1.0, 1.0} and 0.3 < (p.y > 0).mean() < 0.7
    np.testing.assert_allclose(p.X.mean(axis=0), 0.0, atol=1e-6)
    q = synthetic.classification_problem(500, 6, seed=3)
    assert np.array_equal(p.X, q.X) and np.array_equal(p.y, q.y)
    om = synthetic.spectral_draws(2000, 3, seed=1)
    assert om.shape == (2000, 3) and om.flags.c_contiguous
    assert abs(om.mean()) < 0.05 and abs(om.std() - 1.0) < 0.05
    e = synthetic.eeg_shape()
    assert e.X.shape == (14979, 14)
