// Preconditioner state owned by a handle (Sec. 3.1 Nystrom, Sec. 3.3.1 block-Jacobi).
#pragma once

#include <cmath>

#include "kpcg_internal.cuh"

namespace kpcg {

struct PrecondState {
    int kind = KPCG_PREC_NONE;
    bool ready = false;
    int64_t n = 0, m = 0, b = 0;
    double noise = 0.0;
    double jitter = 0.0;
    DevBuf<int64_t> idx;     // inducing rows (Nystrom)
    DevBuf<float> us32;      // scaled inducing rows, FP32
    DevBuf<double> us64;     // scaled inducing rows, FP64
    DevBuf<float2> KXU;      // n x m row-major, FP64 entries as FP32 pairs (hi, lo)
    DevBuf<double> M0;       // sigma^2 K_UU + K_UX K_XU before jitter
    DevBuf<double> M;        // Cholesky factor(s) L
    DevBuf<double> U;        // L^{-T}, row-major (per block for block-Jacobi)
    DevBuf<double> scratch;  // split partials of the set-up products
    DevBuf<double> wpart, w, y;
    DevBuf<int> status;

    void reset() {
        kind = KPCG_PREC_NONE;
        ready = false;
        idx.release();
        us32.release();
        us64.release();
        KXU.release();
        M0.release();
        M.release();
        U.release();
        scratch.release();
        wpart.release();
        w.release();
        y.release();
        status.release();
    }
};

void nystrom_setup(PrecondState& P, const float* xs32, const double* xs64, int64_t n, int dp,
                   float c0_32, double c0_64, double noise, const int64_t* idx_host, int64_t m,
                   cudaStream_t st);
// u = M^{-1} K_UX R (FP64, c columns, u column-major with ld m), the
// coefficient fit of the warm-start basis.
void nystrom_project_solve(const PrecondState& P, const double* R, int64_t ldr, int c, double* u,
                           cudaStream_t st);
// out = K_XU u for one column (FP64).
void nystrom_expand(const PrecondState& P, const double* u, double* out, cudaStream_t st);
void block_jacobi_setup(PrecondState& P, const double* xs64, int64_t n, int dp, double c0_64,
                        double noise, int64_t b, cudaStream_t st);

}  // namespace kpcg
