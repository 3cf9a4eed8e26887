// Preconditioner state owned by a handle (Sec. 3.1 Nystrom, Sec. 3.3.1 block-Jacobi).
#pragma once

#include <cmath>
#include <vector>

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
    double apply_noise = 0.0;  // divisor of the Nystrom apply (1 for FITC's scaled form)
    DevBuf<double> dscale;     // FITC: D^{-1/2}, D = diag(K - Q) + sigma^2
    DevBuf<double> tmp64;      // FITC: scaled right-hand sides
    DevBuf<float> tmp32;
    DevBuf<double> dblk, dinv;  // PITC: block factors L_D of D and U_D = L_D^{-T}

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
        apply_noise = 0.0;
        dscale.release();
        tmp64.release();
        tmp32.release();
        dblk.release();
        dinv.release();
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
// Random-feature preconditioner (Sec. 3.2): P = Phi Phi^T + noise I with
// Phi_i = sqrt(s2/m) [cos(w_r . x~_i), sin(w_r . x~_i)]_r (n x 2m, stored in KXU),
// applied as the Nystrom form with K_UU = I:
// P^{-1} = noise^{-1} [I - Phi (noise I + Phi^T Phi)^{-1} Phi^T].  omega_host:
// m x d standard-normal draws (row-major); in the scaled inputs x~ = (x - mu)/l
// the spectral points s_r = w_r / (2 pi l) act through w_r . x~.
void spectral_setup(PrecondState& P, const double* xs64, int64_t n, int dp, double s2,
                    double noise, const double* omega_host, int d, int64_t m, cudaStream_t st);
// Preconditioner of B = I + W^1/2 K W^1/2 (the Laplace step, Sec. 2.2):
// P_B = I + W^1/2 Q W^1/2 with Q = K_XU K_UU^{-1} K_UX, so
// P_B^{-1} = I - K~ (K_UU + K~^T K~)^{-1} K~^T with K~ = W^1/2 K_XU: the Nystrom
// apply with unit noise on the row-scaled K_XU.  kxu0 keeps the unscaled K_XU
// between Newton steps (computed when `first`); sW = W^1/2 (device, n).
void laplace_precond_setup(PrecondState& P, DevBuf<float2>& kxu0, bool first, const float* xs32,
                           const double* xs64, int64_t n, int dp, double c0_64,
                           const double* sW, const int64_t* idx_host, int64_t m,
                           cudaStream_t st);
void block_jacobi_setup(PrecondState& P, const double* xs64, int64_t n, int dp, double c0_64,
                        double noise, int64_t b, cudaStream_t st);
// FITC (Sec. 3.1): P = Q + diag(K - Q) + sigma^2 I, Q = K_XU K_UU^{-1} K_UX.  With
// D = diag(K - Q) + sigma^2 and K~ = D^{-1/2} K_XU the inversion lemma gives
// P^{-1} = D^{-1/2} [I - K~ (K_UU + K~^T K~)^{-1} K~^T] D^{-1/2}: the Nystrom
// apply with unit noise on the row-scaled K_XU, between two diagonal scalings.
// s2: the amplitude (K_ii = s2).
void fitc_setup(PrecondState& P, const float* xs32, const double* xs64, int64_t n, int dp,
                float c0_32, double c0_64, double s2, double noise, const int64_t* idx_host,
                int64_t m, cudaStream_t st);
// PITC (Sec. 3.1): P = Q + bldiag(K - Q) + sigma^2 I with contiguous blocks of b
// rows.  With D = bldiag(K - Q) + sigma^2 I = L_D L_D^T (block Cholesky) and
// K~ = L_D^{-1} K_XU the inversion lemma gives
// P^{-1} = L_D^{-T} [I - K~ (K_UU + K~^T K~)^{-1} K~^T] L_D^{-1}: the Nystrom apply
// with unit noise between two block-triangular factors.
void pitc_setup(PrecondState& P, const float* xs32, const double* xs64, int64_t n, int dp,
                double c0_64, double noise, const int64_t* idx_host, int64_t m, int64_t b,
                cudaStream_t st);

// ------------------------------------------- batched Nystrom apply
// Problems laid out column by column (problem p owns columns p*c .. p*c+c-1
// of an ld x (P c) block); a single problem is the batch P = 1.
struct NysBatchProb {
    const float2* KXU;  // n x m, FP64 entries as FP32 pairs
    const double* U;    // L^{-T}, m x m row-major
    int64_t n, m;
    int64_t wbase;      // offset of the problem in w / y (c * m doubles)
    int64_t pbase;      // offset of the problem in the split partials
    int32_t nsplit, rows_per_split;
    double inv_noise;
    float inv_noise_f;
};
struct NysBatch {
    int P = 0, c = 0;
    int64_t mmax = 0, wtotal = 0, ptotal = 0;
    int nsplit_max = 0;
    std::vector<NysBatchProb> hprobs;
    DevBuf<NysBatchProb> probs;
    DevBuf<double> part, w, y;
    DevBuf<float2> u2;  // u = M^{-1} K_UX r as FP32 pairs for the back product
    DevBuf<int4> itemsL, itemsU;  // (problem, column, block) items of the triangular applies
    int nL = 0, nU = 0;
};
// Tables for c columns per problem from the problems' Nystrom states
// (problems without one get m = 0 and the identity).
void nys_batch_plan(NysBatch& nb, const std::vector<const PrecondState*>& Ps, int c,
                    cudaStream_t st);
// Z = P_p^{-1} R for every problem (FP32 vectors; FP64 and double-float
// inside), rows n_p .. nrows-1 zero; the columns of problems with no active
// column are skipped and left unchanged.
void nys_batch_apply(NysBatch& nb, const float* R, int64_t ldr, float* Z, int64_t ldz,
                     int64_t nrows, const int* active, cudaStream_t st);

}  // namespace kpcg
