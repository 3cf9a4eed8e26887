"""kpcg: preconditioned conjugate gradients on kernel matrices for GB300.

A thin ctypes binding over ``libkpcg.so`` (the C ABI in ``include/kpcg.h``).
It only marshals arguments: every step of the solve runs in the library's
CUDA kernels.  PyTorch provides device memory and the current stream.  There
is no CPU fallback: if the library or a GPU is missing, the binding raises.
"""
from .binding import (  # noqa: F401
    KPCG_FP32,
    KPCG_DF64,
    KPCG_FP32_IR,
    KPCG_FP32X_IR,
    KPCG_FP64,
    KPCG_PREC_BLOCK_JACOBI,
    KPCG_PREC_FITC,
    KPCG_PREC_NONE,
    KPCG_PREC_NYSTROM,
    KPCG_PREC_PITC,
    KPCG_PREC_SPECTRAL,
    KPCG_TC_IR,
    KPCG_TCX_IR,
    Batch,
    KpcgError,
    LaplaceInfo,
    MLP,
    Options,
    Problem,
    Solver,
    Info,
    default_options,
    exported_symbols,
    fortran_empty,
    lib,
    library_path,
    matvec_f64_noalloc,
    probe_rates,
)
