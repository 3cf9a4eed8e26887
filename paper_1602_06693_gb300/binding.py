"""ctypes binding of the kpcg C ABI (``include/kpcg.h``), same names and arguments.

``lib()`` loads ``libkpcg.so`` (built in-tree by ``build.py``) and raises if
it is missing.  ``Solver`` wraps one handle and takes torch CUDA tensors,
passing their device pointers and the current CUDA stream to the library.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libkpcg.so")

KPCG_PREC_NONE, KPCG_PREC_NYSTROM, KPCG_PREC_BLOCK_JACOBI, KPCG_PREC_FITC = 0, 1, 2, 3
KPCG_PREC_SPECTRAL, KPCG_PREC_PITC = 4, 5
KPCG_FP64, KPCG_FP32, KPCG_FP32_IR, KPCG_TC_IR, KPCG_DF64, KPCG_FP32X_IR, KPCG_TCX_IR = (
    0, 1, 2, 3, 4, 5, 6)

_STATUS = {
    0: "KPCG_OK", 1: "KPCG_ERR_ARG", 2: "KPCG_ERR_CUDA", 3: "KPCG_ERR_OOM",
    4: "KPCG_ERR_NOT_SPD", 5: "KPCG_ERR_BREAKDOWN", 6: "KPCG_ERR_NO_CONVERGENCE",
    7: "KPCG_ERR_TIMEOUT", 8: "KPCG_ERR_STATE",
}

SYMBOLS = (
    "kpcg_default_options", "kpcg_status_string", "kpcg_create", "kpcg_set_theta",
    "kpcg_set_options", "kpcg_precond", "kpcg_matvec_f64", "kpcg_matvec_f32",
    "kpcg_precond_apply_f64", "kpcg_solve", "kpcg_dkv", "kpcg_grad", "kpcg_destroy",
    "kpcg_last_error", "kpcg_matvec_f64_noalloc", "kpcg_predict", "kpcg_warm_basis",
    "kpcg_warm_fit",
    "kpcg_warm_expand", "kpcg_warm_snapshots", "kpcg_warm_push", "kpcg_mlp_create",
    "kpcg_mlp_forward", "kpcg_mlp_grad", "kpcg_mlp_train",
    "kpcg_mlp_get_params", "kpcg_mlp_destroy", "kpcg_mlp_last_error", "kpcg_batch_create",
    "kpcg_batch_solve", "kpcg_batch_matvec_f32", "kpcg_batch_precond_apply_f32",
    "kpcg_batch_tune", "kpcg_batch_set_tiling", "kpcg_batch_set_options", "kpcg_batch_max_n",
    "kpcg_batch_destroy",
    "kpcg_batch_last_error", "kpcg_precond_spectral", "kpcg_laplace", "kpcg_laplace_predict",
    "kpcg_precond_pitc", "kpcg_probe_rates", "kpcg_batch_set_contraction",
)

_NO_STATUS = ("kpcg_destroy", "kpcg_last_error", "kpcg_mlp_destroy", "kpcg_mlp_last_error",
              "kpcg_batch_max_n", "kpcg_batch_destroy", "kpcg_batch_last_error")


class Options(ctypes.Structure):
    _fields_ = [
        ("max_iter", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("tol_mode", ctypes.c_int32),
        ("max_outer", ctypes.c_int32),
        ("inner_tol", ctypes.c_double),
        ("check_every", ctypes.c_int32),
        ("max_restarts", ctypes.c_int32),
        ("inner_shift", ctypes.c_double),
        ("inner_max_iter", ctypes.c_int32),
        ("fcg_window", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("wait_stall", ctypes.c_int32),
        ("wait_limit_ns", ctypes.c_int64),
        ("inner_f64", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("iters_total", ctypes.c_int32),
        ("outer_steps", ctypes.c_int32),
        ("max_rel_res", ctypes.c_double),
        ("time_ms", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("kv_inner_ms", ctypes.c_double),
        ("kv_inner_calls", ctypes.c_int32),
        ("kv_outer_calls", ctypes.c_int32),
        ("kv_outer_ms", ctypes.c_double),
        ("precond_ms", ctypes.c_double),
        ("precond_calls", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("precond_jitter", ctypes.c_double),
        ("resid_ms", ctypes.c_double),
        ("resid_calls", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LaplaceInfo(ctypes.Structure):
    _fields_ = [
        ("newton_steps", ctypes.c_int32),
        ("cg_iters_total", ctypes.c_int32),
        ("psi", ctypes.c_double),
        ("max_rel_res", ctypes.c_double),
        ("time_ms", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("launches", ctypes.c_int32),
        ("precond_builds", ctypes.c_int32),
    ]


class Problem(ctypes.Structure):
    """kpcg_problem: one system of a batch."""
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("ard", ctypes.c_int32), ("log_theta", ctypes.POINTER(ctypes.c_double)),
                ("noise_var", ctypes.c_double), ("m", ctypes.c_int64),
                ("idx", ctypes.POINTER(ctypes.c_int64))]


class KpcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = _STATUS.get(status, str(status))


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libkpcg.so; raise if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build it with `python -m paper_1602_06693_gb300.build` "
                "(the library has no CPU fallback)")
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        pdbl = ctypes.POINTER(ctypes.c_double)
        L.kpcg_default_options.argtypes = [ctypes.POINTER(Options)]
        L.kpcg_default_options.restype = None
        L.kpcg_status_string.argtypes = [ctypes.c_int]
        L.kpcg_status_string.restype = ctypes.c_char_p
        L.kpcg_create.argtypes = [vp, i64, i32, pdbl, i32, dbl, ctypes.POINTER(Options), vp,
                                  ctypes.POINTER(vp)]
        L.kpcg_set_theta.argtypes = [vp, pdbl, dbl]
        L.kpcg_set_options.argtypes = [vp, ctypes.POINTER(Options)]
        L.kpcg_precond.argtypes = [vp, i32, i64, ctypes.POINTER(ctypes.c_int64)]
        L.kpcg_precond_spectral.argtypes = [vp, i64, pdbl]
        L.kpcg_precond_pitc.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int64), i64]
        L.kpcg_laplace.argtypes = [vp, vp, dbl, i32, dbl, vp, vp, ctypes.POINTER(LaplaceInfo)]
        L.kpcg_laplace_predict.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp, dbl,
                                           ctypes.POINTER(LaplaceInfo)]
        L.kpcg_matvec_f64.argtypes = [vp, vp, i64, i32, vp, i64, i32]
        L.kpcg_matvec_f32.argtypes = [vp, vp, i64, i32, vp, i64, i32]
        L.kpcg_precond_apply_f64.argtypes = [vp, vp, i64, i32, vp, i64]
        L.kpcg_solve.argtypes = [vp, vp, i64, i32, dbl, vp, vp, i64,
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(Info)]
        L.kpcg_dkv.argtypes = [vp, vp, i64, i32, vp, i64]
        L.kpcg_grad.argtypes = [vp, vp, vp, i32, dbl, vp, pdbl, vp, ctypes.POINTER(Info)]
        L.kpcg_predict.argtypes = [vp, vp, i64, vp, vp, vp, dbl, ctypes.POINTER(Info)]
        L.kpcg_warm_basis.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int64), dbl]
        L.kpcg_warm_snapshots.argtypes = [vp, i32, dbl]
        L.kpcg_warm_push.argtypes = [vp, vp]
        L.kpcg_warm_fit.argtypes = [vp, vp, vp]
        L.kpcg_warm_expand.argtypes = [vp, vp, vp]
        pflt = ctypes.POINTER(ctypes.c_float)
        L.kpcg_mlp_create.argtypes = [i32, i32, i32, i32, pflt, i32, vp, ctypes.POINTER(vp)]
        L.kpcg_mlp_forward.argtypes = [vp, vp, i32, vp, i32]
        L.kpcg_mlp_grad.argtypes = [vp, vp, vp, i32, vp, pflt]
        L.kpcg_mlp_train.argtypes = [vp, vp, vp, i32, i32, ctypes.c_float, pflt]
        L.kpcg_mlp_get_params.argtypes = [vp, pflt]
        L.kpcg_mlp_destroy.argtypes = [vp]
        L.kpcg_mlp_destroy.restype = None
        L.kpcg_mlp_last_error.argtypes = [vp]
        L.kpcg_mlp_last_error.restype = ctypes.c_char_p
        L.kpcg_matvec_f64_noalloc.argtypes = [vp, i64, i32, pdbl, i32, dbl, vp, i64, i32, vp,
                                              i64, vp]
        L.kpcg_probe_rates.argtypes = [vp, pdbl]
        L.kpcg_batch_create.argtypes = [i32, ctypes.POINTER(Problem), ctypes.POINTER(Options), vp,
                                        ctypes.POINTER(vp)]
        L.kpcg_batch_solve.argtypes = [vp, vp, i64, i32, dbl, vp, ctypes.POINTER(ctypes.c_int32),
                                       pdbl, ctypes.POINTER(Info)]
        L.kpcg_batch_matvec_f32.argtypes = [vp, vp, i64, i32, vp]
        L.kpcg_batch_precond_apply_f32.argtypes = [vp, vp, i64, i32, vp]
        L.kpcg_batch_tune.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), pflt]
        L.kpcg_batch_set_tiling.argtypes = [vp, i32, i32]
        L.kpcg_batch_set_contraction.argtypes = [vp, i32]
        L.kpcg_batch_set_options.argtypes = [vp, ctypes.POINTER(Options)]
        L.kpcg_batch_max_n.argtypes = [vp]
        L.kpcg_batch_max_n.restype = ctypes.c_int64
        L.kpcg_batch_destroy.argtypes = [vp]
        L.kpcg_batch_destroy.restype = None
        L.kpcg_batch_last_error.argtypes = [vp]
        L.kpcg_batch_last_error.restype = ctypes.c_char_p
        L.kpcg_destroy.argtypes = [vp]
        L.kpcg_destroy.restype = None
        L.kpcg_last_error.argtypes = [vp]
        L.kpcg_last_error.restype = ctypes.c_char_p
        for name in SYMBOLS[2:]:
            if name not in _NO_STATUS:
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def exported_symbols():
    """Names from include/kpcg.h that the loaded library exports."""
    L = lib()
    return [s for s in SYMBOLS if hasattr(L, s)]


def matvec_f64_noalloc(X, log_theta, noise, V, ard=True, out=None, stream=None):
    """kpcg_matvec_f64_noalloc: (K + noise I) V in FP64 without device allocation
    inside the library (its scratch is a static device array)."""
    torch = _torch()
    if X.dtype != torch.float32 or not X.is_cuda or not X.is_contiguous():
        raise TypeError("X must be a contiguous float32 CUDA tensor (n x d row-major)")
    n, d = int(X.shape[0]), int(X.shape[1])
    V, ldv, c = _colmajor(V, "V")
    O = out if out is not None else (torch.empty_like(V) if V.dim() == 1 else
                                     fortran_empty(n, c, torch.float64, V.device))
    O_, ldo, co = _colmajor(O, "out")
    if tuple(O.shape) != tuple(V.shape) or O.device != V.device:
        raise ValueError("out must have V's shape and device")
    if co != c:
        raise ValueError("out must have as many columns as V")
    lt = np.ascontiguousarray(log_theta, dtype=np.float64)
    st = stream if stream is not None else torch.cuda.current_stream(X.device)
    L = lib()
    rc = L.kpcg_matvec_f64_noalloc(ctypes.c_void_p(X.data_ptr()), n, d,
                                   lt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(ard),
                                   float(noise), _dptr(V, torch.float64, "V"), ldv, c,
                                   _dptr(O_, torch.float64, "out"), ldo,
                                   ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise KpcgError(rc, L.kpcg_last_error(None).decode())
    return O


def probe_rates(stream=None):
    """kpcg_probe_rates: measured FP32 FMA, MUFU ex2 and FP64 FMA lane-instruction
    rates (per second) of the current device, the SM clock (MHz) inside each
    probe, and the SM count."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    out = (ctypes.c_double * 7)()
    L = lib()
    rc = L.kpcg_probe_rates(ctypes.c_void_p(st.cuda_stream), out)
    if rc != 0:
        raise KpcgError(rc, L.kpcg_last_error(None).decode())
    v = list(out)
    return {"fp32_fma_per_s": v[0], "ex2_per_s": v[1], "fp64_fma_per_s": v[2],
            "sm_mhz_fp32": v[3], "sm_mhz_ex2": v[4], "sm_mhz_fp64": v[5], "sms": int(v[6])}


def default_options(**kw) -> Options:
    o = Options()
    lib().kpcg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _torch():
    import torch
    return torch


def _dptr(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _colmajor(t, name):
    """(ptr-able tensor, ld, c) for a 1-D or column-major 2-D tensor."""
    if t.dim() == 1:
        return t, t.shape[0], 1
    if t.dim() == 2 and t.stride(0) == 1:
        return t, t.stride(1) if t.shape[1] > 1 else t.shape[0], t.shape[1]
    raise ValueError(f"{name} must be 1-D or column-major 2-D (use .t().contiguous().t())")


def fortran_empty(n, c, dtype, device):
    """n x c column-major CUDA tensor."""
    torch = _torch()
    return torch.empty((c, n), dtype=dtype, device=device).t()


class Solver:
    """One kpcg handle (kpcg_create ... kpcg_destroy) bound to the current stream."""

    def __init__(self, X, log_theta, noise, ard=True, options: Options | None = None,
                 stream=None):
        torch = _torch()
        L = lib()
        if X.dtype != torch.float32 or not X.is_cuda or not X.is_contiguous():
            raise TypeError("X must be a contiguous float32 CUDA tensor (n x d row-major)")
        self.n, self.d = int(X.shape[0]), int(X.shape[1])
        self.ard = bool(ard)
        self.device = X.device
        lt = np.ascontiguousarray(log_theta, dtype=np.float64)
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        opt = options if options is not None else default_options()
        self.options = opt
        st = L.kpcg_create(ctypes.c_void_p(X.data_ptr()), self.n, self.d,
                           lt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(self.ard),
                           float(noise), ctypes.byref(opt),
                           ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise KpcgError(st, L.kpcg_last_error(None).decode())
        self._h = h

    # -- plumbing
    def _check(self, st):
        if st != 0:
            raise KpcgError(st, lib().kpcg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().kpcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def n_theta(self):
        return (self.d if self.ard else 1) + 1

    # -- API
    def set_theta(self, log_theta, noise):
        lt = np.ascontiguousarray(log_theta, dtype=np.float64)
        self._check(lib().kpcg_set_theta(self._h, lt.ctypes.data_as(
            ctypes.POINTER(ctypes.c_double)), float(noise)))

    def set_options(self, options: Options):
        self.options = options
        self._check(lib().kpcg_set_options(self._h, ctypes.byref(options)))

    def precond(self, kind, size=0, idx=None):
        p = None
        if idx is not None:
            idx = np.ascontiguousarray(idx, dtype=np.int64)
            p = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        self._check(lib().kpcg_precond(self._h, int(kind), int(size), p))

    def precond_pitc(self, m, idx, b):
        """PITC preconditioner (Sec. 3.1): m inducing rows idx, blocks of b rows."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        self._check(lib().kpcg_precond_pitc(self._h, int(m),
                                            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                            int(b)))

    def precond_spectral(self, omega):
        """Random-feature preconditioner (Sec. 3.2) from m x d standard-normal draws."""
        om = np.ascontiguousarray(omega, dtype=np.float64).reshape(-1, self.d)
        self._check(lib().kpcg_precond_spectral(
            self._h, int(om.shape[0]), om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def laplace(self, y, newton_tol=1e-12, max_newton=50, cg_tol=1e-10, want_a=True):
        """Probit Laplace mode (Sec. 2.2, Appendix B): returns (f, a, info, status);
        y is a float64 CUDA vector of +-1 labels."""
        torch = _torch()
        if y.dtype != torch.float64 or not y.is_cuda or y.dim() != 1 or not y.is_contiguous():
            raise TypeError("y must be a contiguous float64 CUDA vector")
        f = torch.empty(self.n, dtype=torch.float64, device=y.device)
        a = torch.empty(self.n, dtype=torch.float64, device=y.device) if want_a else None
        info = LaplaceInfo()
        st = lib().kpcg_laplace(self._h, ctypes.c_void_p(y.data_ptr()), float(newton_tol),
                                int(max_newton), float(cg_tol), ctypes.c_void_p(f.data_ptr()),
                                ctypes.c_void_p(a.data_ptr()) if a is not None else None,
                                ctypes.byref(info))
        if st not in (0, 6):
            self._check(st)
        return f, a, info, st

    def laplace_predict(self, y, f, a, Xs, var=True, prob=True, cg_tol=1e-10):
        """Probit predictions at Xs (float32 CUDA, ns x d) from the mode (f, a):
        returns (mean, var or None, prob or None, LaplaceInfo)."""
        torch = _torch()
        if Xs.dtype != torch.float32 or not Xs.is_cuda or not Xs.is_contiguous():
            raise TypeError("Xs must be a contiguous float32 CUDA tensor (ns x d row-major)")
        ns = int(Xs.shape[0])
        mk = lambda: torch.empty(ns, dtype=torch.float64, device=Xs.device)  # noqa: E731
        mean = mk()
        v = mk() if var else None
        p = mk() if prob else None
        info = LaplaceInfo()
        f64 = torch.float64
        for t, nm in ((y, "y"), (f, "f"), (a, "a")):
            if t.dim() != 1 or t.shape[0] != self.n or not t.is_contiguous():
                raise TypeError(f"{nm} must be a contiguous vector of length n")
        self._check(lib().kpcg_laplace_predict(
            self._h, _dptr(y, f64, "y"), _dptr(f, f64, "f"), _dptr(a, f64, "a"),
            ctypes.c_void_p(Xs.data_ptr()), ns, _dptr(mean, f64, "mean"),
            _dptr(v, f64, "var") if v is not None else None,
            _dptr(p, f64, "prob") if p is not None else None, float(cg_tol),
            ctypes.byref(info)))
        return mean, v, p, info

    def matvec_f64(self, V, impl=0, out=None):
        torch = _torch()
        V, ldv, c = _colmajor(V, "V")
        O = out if out is not None else (torch.empty_like(V) if V.dim() == 1 else
                                         fortran_empty(self.n, c, torch.float64, V.device))
        O_, ldo, _ = _colmajor(O, "out")
        self._check(lib().kpcg_matvec_f64(self._h, _dptr(V, torch.float64, "V"), ldv, c,
                                          _dptr(O_, torch.float64, "out"), ldo, int(impl)))
        return O

    def matvec_f32(self, V, impl=0, out=None):
        torch = _torch()
        V, ldv, c = _colmajor(V, "V")
        O = out if out is not None else (torch.empty_like(V) if V.dim() == 1 else
                                         fortran_empty(self.n, c, torch.float32, V.device))
        O_, ldo, _ = _colmajor(O, "out")
        self._check(lib().kpcg_matvec_f32(self._h, _dptr(V, torch.float32, "V"), ldv, c,
                                          _dptr(O_, torch.float32, "out"), ldo, int(impl)))
        return O

    def precond_apply(self, R):
        torch = _torch()
        R, ldr, c = _colmajor(R, "R")
        Z = torch.empty_like(R) if R.dim() == 1 else fortran_empty(self.n, c, torch.float64,
                                                                  R.device)
        Z_, ldz, _ = _colmajor(Z, "Z")
        self._check(lib().kpcg_precond_apply_f64(self._h, _dptr(R, torch.float64, "R"), ldr, c,
                                                 _dptr(Z_, torch.float64, "Z"), ldz))
        return Z

    def solve(self, B, tol=1e-8, X0=None, raise_on_error=True):
        """Solve K_y X = B; returns (X, iters per column, Info, status)."""
        torch = _torch()
        B, ldb, c = _colmajor(B, "B")
        X = torch.empty_like(B) if B.dim() == 1 else fortran_empty(self.n, c, torch.float64,
                                                                  B.device)
        X_, ldx, _ = _colmajor(X, "X")
        x0p = None
        if X0 is not None:
            X0_, ldx0, _ = _colmajor(X0, "X0")
            if ldx0 != ldx:
                X0_ = X0_.clone() if X0_.dim() == 1 else X0_.t().contiguous().t()
            x0p = _dptr(X0_, torch.float64, "X0")
        iters = (ctypes.c_int32 * c)()
        info = Info()
        st = lib().kpcg_solve(self._h, _dptr(B, torch.float64, "B"), ldb, c, float(tol), x0p,
                              _dptr(X_, torch.float64, "X"), ldx, iters, ctypes.byref(info))
        if st != 0 and raise_on_error:
            self._check(st)
        return X, np.array(list(iters), dtype=np.int64), info, st

    def dkv(self, W):
        torch = _torch()
        W, ldw, c = _colmajor(W, "W")
        G = torch.empty((self.n_theta, c, self.n), dtype=torch.float64, device=W.device)
        self._check(lib().kpcg_dkv(self._h, _dptr(W, torch.float64, "W"), ldw, c,
                                   ctypes.c_void_p(G.data_ptr()), self.n))
        return G.transpose(1, 2)  # (n_theta, n, c)

    def grad(self, y, probes, tol=1e-8, want_alpha=False, alpha0=None):
        """Stochastic gradient of log p (Eq. 2): returns (grad[n_theta+1], alpha|None, Info)."""
        torch = _torch()
        if y.dim() != 1 or not y.is_contiguous():
            raise ValueError("y must be a contiguous 1-D tensor")
        P, ldp, t = _colmajor(probes, "probes")
        if ldp != self.n:
            raise ValueError("probes must have leading dimension n")
        g = np.zeros(self.n_theta + 1, dtype=np.float64)
        alpha = torch.empty(self.n, dtype=torch.float64, device=y.device) if want_alpha else None
        info = Info()
        a0 = _dptr(alpha0, torch.float64, "alpha0") if alpha0 is not None else None
        self._check(lib().kpcg_grad(self._h, _dptr(y, torch.float64, "y"),
                                    _dptr(P, torch.float64, "probes"), t, float(tol), a0,
                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    _dptr(alpha, torch.float64, "alpha") if want_alpha else None,
                                    ctypes.byref(info)))
        return g, alpha, info

    def predict(self, Xs, alpha, var=True, tol=1e-10):
        """Predictive mean and latent variance at test inputs Xs (float32 CUDA,
        ns x d): returns (mean, var | None, Info)."""
        torch = _torch()
        Xs = Xs.contiguous()
        if Xs.dtype != torch.float32 or Xs.dim() != 2:
            raise ValueError("Xs must be a float32 (ns, d) tensor")
        ns = Xs.shape[0]
        mean = torch.empty(ns, dtype=torch.float64, device=Xs.device)
        v = torch.empty(ns, dtype=torch.float64, device=Xs.device) if var else None
        info = Info()
        self._check(lib().kpcg_predict(self._h, _dptr(Xs, torch.float32, "Xs"), ns,
                                       _dptr(alpha, torch.float64, "alpha"),
                                       _dptr(mean, torch.float64, "mean"),
                                       _dptr(v, torch.float64, "var") if var else None,
                                       float(tol), ctypes.byref(info)))
        return mean, v, info

    # -- learned warm start: basis fit and expansion
    def warm_basis(self, idx, ridge=1e-6):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        self.m_warm = int(idx.shape[0])
        self._check(lib().kpcg_warm_basis(self._h, self.m_warm,
                                          idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          float(ridge)))

    def warm_snapshots(self, q, ridge=1e-10):
        self.m_warm = int(q)
        self._check(lib().kpcg_warm_snapshots(self._h, int(q), float(ridge)))

    def warm_push(self, a):
        torch = _torch()
        self._check(lib().kpcg_warm_push(self._h, _dptr(a, torch.float64, "a")))

    def warm_fit(self, a):
        torch = _torch()
        c = torch.empty(self.m_warm, dtype=torch.float64, device=a.device)
        self._check(lib().kpcg_warm_fit(self._h, _dptr(a, torch.float64, "a"),
                                        _dptr(c, torch.float64, "c")))
        return c

    def warm_expand(self, c):
        torch = _torch()
        x0 = torch.empty(self.n, dtype=torch.float64, device=c.device)
        self._check(lib().kpcg_warm_expand(self._h, _dptr(c, torch.float64, "c"),
                                           _dptr(x0, torch.float64, "x0")))
        return x0


MLP_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


class MLP:
    """The warm-start network (kpcg_mlp_*): parameters live on the GPU."""

    def __init__(self, params: dict, max_batch=256, stream=None):
        torch = _torch()
        self.shapes = {k: np.asarray(params[k]).shape for k in MLP_NAMES}
        h1, n_in = self.shapes["W1"]
        h2 = self.shapes["W2"][0]
        n_out = self.shapes["W3"][0]
        self.dims = (n_in, h1, h2, n_out)
        flat = np.concatenate([np.asarray(params[k], dtype=np.float32).ravel() for k in MLP_NAMES])
        self.size = flat.size
        st = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        L = lib()
        rc = L.kpcg_mlp_create(n_in, h1, h2, n_out,
                               flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(max_batch),
                               ctypes.c_void_p(st.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise KpcgError(rc, L.kpcg_mlp_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != 0:
            raise KpcgError(rc, lib().kpcg_mlp_last_error(self._h).decode())

    def forward(self, X, bf16=False):
        torch = _torch()
        X = X.contiguous()
        out = torch.empty((X.shape[0], self.dims[3]), dtype=torch.float32, device=X.device)
        self._check(lib().kpcg_mlp_forward(self._h, _dptr(X, torch.float32, "X"), X.shape[0],
                                           _dptr(out, torch.float32, "out"), int(bool(bf16))))
        return out

    def grad(self, X, T):
        torch = _torch()
        g = torch.empty(self.size, dtype=torch.float32, device=X.device)
        loss = ctypes.c_float()
        self._check(lib().kpcg_mlp_grad(self._h, _dptr(X, torch.float32, "X"),
                                        _dptr(T, torch.float32, "T"), X.shape[0],
                                        _dptr(g, torch.float32, "g"), ctypes.byref(loss)))
        return self._unflatten(g.cpu().numpy()), float(loss.value)

    def train(self, X, T, epochs, lr):
        """Full-batch Adam; X and T must stay alive while trained with (graph)."""
        torch = _torch()
        loss = ctypes.c_float()
        self._keep = (X, T)
        self._check(lib().kpcg_mlp_train(self._h, _dptr(X, torch.float32, "X"),
                                         _dptr(T, torch.float32, "T"), X.shape[0], int(epochs),
                                         float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def params(self):
        flat = np.empty(self.size, dtype=np.float32)
        self._check(lib().kpcg_mlp_get_params(self._h,
                                              flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return self._unflatten(flat)

    def _unflatten(self, flat):
        out, o = {}, 0
        for k in MLP_NAMES:
            sz = int(np.prod(self.shapes[k]))
            out[k] = flat[o:o + sz].reshape(self.shapes[k])
            o += sz
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().kpcg_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent systems of uneven size (kpcg_batch_*).

    problems: sequence of (X, log_theta, noise, idx) with X a (n_p, d_p) float32
    CUDA tensor and idx the sorted inducing rows (None: no preconditioner).
    Block tensors are (ld, P*c) column-major float64/float32 CUDA tensors with
    ld = max_n; ``block``/``unblock`` convert from/to per-problem (n_p, c) arrays.
    """

    def __init__(self, problems, ard=True, options: Options | None = None, stream=None):
        torch = _torch()
        self._keep = []
        arr = (Problem * len(problems))()
        self.ns = []
        for k, (X, log_theta, noise, idx) in enumerate(problems):
            X = X.contiguous()
            if X.dtype != torch.float32 or not X.is_cuda:
                raise ValueError("X must be a float32 CUDA tensor")
            lt = np.ascontiguousarray(log_theta, dtype=np.float64)
            ix = None if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
            self._keep += [X, lt, ix]
            arr[k].X = X.data_ptr()
            arr[k].n = X.shape[0]
            arr[k].d = X.shape[1]
            arr[k].ard = 1 if ard else 0
            arr[k].log_theta = lt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[k].noise_var = float(noise)
            arr[k].m = 0 if ix is None else ix.shape[0]
            arr[k].idx = (ix.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if ix is not None
                          else ctypes.POINTER(ctypes.c_int64)())
            self.ns.append(int(X.shape[0]))
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        h = ctypes.c_void_p()
        L = lib()
        rc = L.kpcg_batch_create(len(problems), arr,
                                 ctypes.byref(options) if options is not None else None,
                                 ctypes.c_void_p(st.cuda_stream), ctypes.byref(h))
        self._keep = None
        if rc != 0:
            raise KpcgError(rc, L.kpcg_batch_last_error(None).decode())
        self._h = h
        self.P = len(problems)
        self.ld = int(L.kpcg_batch_max_n(h))

    def _check(self, rc):
        if rc != 0:
            raise KpcgError(rc, lib().kpcg_batch_last_error(self._h).decode())

    def empty(self, c, dtype):
        torch = _torch()
        return torch.zeros((self.P * c, self.ld), dtype=dtype, device="cuda").t()

    def block(self, vectors, dtype=None):
        """Per-problem (n_p, c) arrays/tensors -> (ld, P*c) column-major block."""
        torch = _torch()
        c = vectors[0].shape[1] if vectors[0].ndim == 2 else 1
        dtype = dtype or torch.float64
        out = self.empty(c, dtype)
        for p, v in enumerate(vectors):
            t = torch.as_tensor(np.asarray(v) if not torch.is_tensor(v) else v).to(
                device="cuda", dtype=dtype).reshape(self.ns[p], c)
            out[: self.ns[p], p * c:(p + 1) * c] = t
        return out

    def unblock(self, Bk, c):
        return [Bk[: self.ns[p], p * c:(p + 1) * c] for p in range(self.P)]

    def _blk(self, T, c, dtype, name):
        torch = _torch()
        if T.dtype != dtype or T.stride(0) != 1 or T.shape[1] != self.P * c or T.shape[0] < self.ld:
            raise ValueError(f"{name} must be a column-major ({self.ld}, {self.P * c}) {dtype} block")
        return T.data_ptr(), T.stride(1)

    def solve(self, B, c, tol=1e-8, raise_on_error=True):
        """Returns (X block, iters (P, c), rel_res (P, c), Info, status)."""
        torch = _torch()
        pb, ld = self._blk(B, c, torch.float64, "B")
        X = torch.zeros((self.P * c, ld), dtype=torch.float64, device="cuda").t()
        it = (ctypes.c_int32 * (self.P * c))()
        rel = (ctypes.c_double * (self.P * c))()
        info = Info()
        rc = lib().kpcg_batch_solve(self._h, pb, ld, c, float(tol), X.data_ptr(), it, rel,
                                    ctypes.byref(info))
        if rc != 0 and raise_on_error:
            self._check(rc)
        return (X, np.array(list(it)).reshape(self.P, c), np.array(list(rel)).reshape(self.P, c),
                info, rc)

    def matvec_f32(self, V, c):
        torch = _torch()
        pv, ld = self._blk(V, c, torch.float32, "V")
        O = torch.zeros((self.P * c, ld), dtype=torch.float32, device="cuda").t()
        self._check(lib().kpcg_batch_matvec_f32(self._h, pv, ld, c, O.data_ptr()))
        return O

    def precond_apply_f32(self, R, c):
        torch = _torch()
        pr, ld = self._blk(R, c, torch.float32, "R")
        Z = torch.zeros((self.P * c, ld), dtype=torch.float32, device="cuda").t()
        self._check(lib().kpcg_batch_precond_apply_f32(self._h, pr, ld, c, Z.data_ptr()))
        return Z

    def tune(self, c):
        g, n, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        self._check(lib().kpcg_batch_tune(self._h, c, ctypes.byref(g), ctypes.byref(n),
                                          ctypes.byref(ms)))
        return int(g.value), int(n.value), float(ms.value)

    def set_options(self, options: Options):
        self._check(lib().kpcg_batch_set_options(self._h, ctypes.byref(options)))

    def set_tiling(self, tiles_per_item, ctas=0):
        self._check(lib().kpcg_batch_set_tiling(self._h, int(tiles_per_item), int(ctas)))

    def set_contraction(self, mode):
        """-1 autotuner's choice, 0 FP32 FMAs, 1 tensor cores (kpcg_batch_set_contraction)."""
        self._check(lib().kpcg_batch_set_contraction(self._h, int(mode)))

    def close(self):
        if getattr(self, "_h", None):
            lib().kpcg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
