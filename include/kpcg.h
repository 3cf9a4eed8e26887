/*
 * kpcg.h -- C ABI of the GB300 library for preconditioned conjugate gradients
 * on kernel matrices, after Cutajar, Osborne, Cunningham and Filippone,
 * "Preconditioning Kernel Matrices" (ICML 2016).
 *
 * The library solves (K(X,X|theta) + sigma^2 I) alpha = B for a block of
 * right-hand sides (Sec. 2.1, Algorithm 1) with the RBF/ARD kernel of Eq. 1,
 * preconditioned by the Nystrom, FITC or PITC (Sec. 3.1), random-feature
 * (Sec. 3.2) or block-Jacobi (Sec. 3.3.1) approximation, estimates the
 * gradient of the log marginal likelihood (Eq. 2) with Rademacher probes
 * (Sec. 2.1), predicts at test inputs, solves many uneven problems in one
 * batch, and finds the Laplace approximation of probit GP classification
 * (Sec. 2.2, Appendix B) with its predictions.  K is never stored: its
 * entries are rebuilt from X inside every product.
 *
 * Notation: amplitude s^2 (the paper's sigma^2 in Eq. 1), noise sigma^2 (the
 * paper's lambda), lengthscales l_r.  Parameters are passed in log space:
 *   ARD:       log_theta = [log l_1, ..., log l_d, log s^2]   (d+1 values)
 *   isotropic: log_theta = [log l, log s^2]                    (2 values)
 *
 * Conventions shared by every entry point
 *   - Every function returns a kpcg_status; KPCG_OK is 0.  On error the
 *     message is available from kpcg_last_error(h) until the next call on h.
 *   - Pointers are DEVICE pointers unless the argument says "host".
 *   - Block vectors are column-major: column k of B starts at B + k*ldb,
 *     ldb >= n.  Device pointers of doubles must be 8-byte aligned.
 *   - The caller owns every buffer it passes; the library copies X at
 *     kpcg_create and owns its own workspaces, released by kpcg_destroy.
 *   - A handle is bound to the CUDA device current at kpcg_create and to the
 *     stream given there; all work is enqueued on that stream and every call
 *     returns after the stream has finished the call's work.  Handles are not
 *     thread-safe; distinct handles may be used from distinct threads.
 *   - No call falls back to the CPU: a missing or failing GPU is an error.
 */
#ifndef KPCG_H
#define KPCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kpcg_ctx* kpcg_t;

typedef enum {
    KPCG_OK = 0,
    KPCG_ERR_ARG = 1,            /* invalid argument (sizes, NULL, alignment)   */
    KPCG_ERR_CUDA = 2,           /* a CUDA runtime call failed                  */
    KPCG_ERR_OOM = 3,            /* device allocation failed                    */
    KPCG_ERR_NOT_SPD = 4,        /* a factorization met a non-positive pivot    */
    KPCG_ERR_BREAKDOWN = 5,      /* p^T K_y p <= 0 or NaN inside CG             */
    KPCG_ERR_NO_CONVERGENCE = 6, /* tolerance not met within the limits         */
    KPCG_ERR_TIMEOUT = 7,        /* a bounded device wait expired               */
    KPCG_ERR_STATE = 8           /* call out of order (e.g. no preconditioner)  */
} kpcg_status;

typedef enum {
    KPCG_PREC_NONE = 0,          /* P = I: plain CG                              */
    KPCG_PREC_NYSTROM = 1,       /* P = K_XU K_UU^-1 K_UX + sigma^2 I (Sec. 3.1)  */
    KPCG_PREC_BLOCK_JACOBI = 2,  /* P = bldiag(K_y) (Sec. 3.3.1)                  */
    KPCG_PREC_FITC = 3,          /* P = Q + diag(K - Q) + sigma^2 I, Q the Nystrom
                                    approximation K_XU K_UU^-1 K_UX (Sec. 3.1)   */
    KPCG_PREC_SPECTRAL = 4,      /* P = Phi Phi^T + sigma^2 I, random Fourier
                                    features (Sec. 3.2); kpcg_precond_spectral   */
    KPCG_PREC_PITC = 5           /* P = Q + bldiag(K - Q) + sigma^2 I (Sec. 3.1);
                                    kpcg_precond_pitc                             */
} kpcg_precond_kind;

typedef enum {
    KPCG_FP64 = 0,     /* FP64 entries, vectors and scalars throughout           */
    KPCG_FP32 = 1,     /* plain FP32 PCG: FP32 entries (direct differences),
                          FP32 vectors; no refinement                            */
    KPCG_FP32_IR = 2,  /* mixed: outer flexible CG (Notay) in FP64 whose
                          preconditioner is an inner FP32 PCG on the shifted
                          operator K + sigma^2 (1 + inner_shift) I               */
    KPCG_TC_IR = 3,    /* as KPCG_FP32_IR, the inner K.V on the tensor cores:
                          tcgen05 BF16 MMAs on a three-way split of the scaled
                          inputs form the exponent in FP32 (TMEM), exp2 on the
                          MUFU; requires d <= 20                                 */
    KPCG_DF64 = 4,     /* FP64 vectors and scalars; iterations use the
                          double-float K.V (FP32-pair arithmetic on the FP32
                          pipe, about 44 bits); stop and restart decisions use
                          the native FP64 residual                               */
    KPCG_FP32X_IR = 5, /* as KPCG_FP32_IR, the inner K.V in FP32 on exact
                          pairwise differences: the scaled inputs stay split
                          into FP32 pairs (no per-point rounding), each entry
                          rounds once in FP32, row and column sums are
                          compensated; requires d <= 16                          */
    KPCG_TCX_IR = 6    /* as KPCG_TC_IR, the inner K.V on per-point-exact
                          tensor-core operands: the scaled inputs cut into five
                          8-bit BF16 slices, the exponent summed level by level
                          (FP32 roundings relative to the exponent itself),
                          exp2 on the MUFU, compensated row sums; d <= 10       */
} kpcg_precision;

typedef struct {
    int32_t max_iter;     /* CG iterations per solve (all inner ones in mixed
                             modes); default 100000 (the paper's cap, Sec. 4)  */
    int32_t precision;    /* kpcg_precision; default KPCG_FP32_IR              */
    int32_t tol_mode;     /* 0: ||b - K_y x|| <= tol ||b|| per column (default);
                             1: the paper's absolute ||r||^2 < n*tol (Sec. 4)  */
    int32_t max_outer;    /* outer flexible-CG steps in mixed modes; def. 60   */
    double inner_tol;     /* relative residual reduction asked of each inner
                             solve in mixed modes; default 1e-2               */
    int32_t check_every;  /* host polls convergence every k iterations; def. 4 */
    int32_t max_restarts; /* residual-replacement restarts in single-precision
                             modes; default 5                                  */
    double inner_shift;   /* mixed modes: the inner operator and the
                             preconditioner use noise sigma^2 (1 + inner_shift),
                             which keeps the reduced-precision inner system
                             positive definite; default 1.0                    */
    int32_t inner_max_iter; /* CG iterations per inner solve; default 2000    */
    int32_t fcg_window;   /* A-orthogonal directions kept by the outer
                             flexible CG; default 16                           */
    int32_t profile;      /* 1: time every K.V and preconditioner call with CUDA
                             events on the handle's stream and report the sums
                             in kpcg_info; default 0                           */
    int32_t wait_stall;   /* test hook of the bounded waits: 1 makes the MMA
                             thread of the single-problem tensor-core kernels
                             first wait on a barrier nothing arrives at, so the
                             wait expires and the call returns KPCG_ERR_TIMEOUT;
                             default 0                                          */
    int64_t wait_limit_ns; /* limit of each wait inside the tensor-core kernels
                             (ns); 0 = the default, 2 s; a wait that expires
                             records an error, lets the kernel's own bulk copies
                             land, frees its tensor memory and returns          */
    int32_t inner_f64;    /* KPCG_TCX_IR: 1 runs the inner PCG on FP64 vectors
                             (the sliced tensor-core product takes them as FP32
                             pairs and returns FP64), so the inner solve is
                             limited by the operator, not by FP32 vectors;
                             default 0                                          */
} kpcg_options;

typedef struct {
    int32_t iters_total;  /* CG iterations run (sum over inner solves)          */
    int32_t outer_steps;  /* outer flexible-CG steps (mixed modes), else restarts */
    double max_rel_res;   /* max over columns of ||b - K_y x|| / ||b||,
                             recomputed in FP64 on the device at return        */
    double time_ms;       /* wall time of the call on the host                  */
    double setup_ms;      /* part of time_ms spent in preconditioner set-up     */
    /* Filled when opt.profile = 1 (device time from CUDA events), else 0:     */
    double kv_inner_ms;   /* reduced-precision K.V calls (mixed modes) or the
                             working-precision K.V calls (single modes)        */
    int32_t kv_inner_calls;
    int32_t kv_outer_calls;
    double kv_outer_ms;   /* double-float K.V calls of the outer loop's
                             directions (mixed modes)                          */
    double precond_ms;    /* preconditioner applications                       */
    int32_t precond_calls;
    int32_t launches;     /* CUDA kernels this call launched (always filled)   */
    double precond_jitter; /* diagonal jitter the Nystrom inner matrix needed
                             (0 when it factored as built)                    */
    double resid_ms;      /* (profile = 1) true-residual products: the native
                             FP64 certifications and double-float steering
                             residuals                                         */
    int32_t resid_calls;
} kpcg_info;

/* Fill *opt with the defaults documented in kpcg_options. */
void kpcg_default_options(kpcg_options* opt);

/* Human-readable name of a status code (static string). */
const char* kpcg_status_string(kpcg_status s);

/* Create a handle for the n x d inputs X (device, float32, row-major,
 * borrowed for the duration of the call and copied).  log_theta (host) holds
 * d+1 (ard != 0) or 2 (ard == 0) log parameters as described above;
 * noise_var is sigma^2 > 0.  opt may be NULL (defaults).  stream is a
 * cudaStream_t (NULL = the legacy default stream).  Supports 1 <= d <= 32.
 * Eq. 1 defines the kernel; Sec. 2.1 defines K_y = K + sigma^2 I. */
kpcg_status kpcg_create(const float* X, int64_t n, int32_t d, const double* log_theta,
                        int32_t ard, double noise_var, const kpcg_options* opt,
                        void* stream, kpcg_t* out);

/* Replace the hyperparameters (host log_theta, same length as at create).
 * The preconditioner is rebuilt for the new theta, from the last
 * kpcg_precond request, at the next call that needs it. */
kpcg_status kpcg_set_theta(kpcg_t h, const double* log_theta, double noise_var);

/* Replace the options (host struct). */
kpcg_status kpcg_set_options(kpcg_t h, const kpcg_options* opt);

/* Build the preconditioner for the current theta.
 *   KPCG_PREC_NYSTROM: size = m, idx (host, m distinct sorted row indices of X)
 *     names the inducing points U (Sec. 3.1; the paper draws them at random
 *     from X, Sec. 5).  P^-1 = sigma^-2 [I - K_XU (sigma^2 K_UU + K_UX K_XU)^-1
 *     K_UX], the inversion lemma applied to P (the printed form drops the
 *     sigma^2 on K_UU).  If the inner matrix is not positive definite, jitter
 *     1e-12*tr/m*10^k (k = 0..6) is added to its diagonal.
 *   KPCG_PREC_BLOCK_JACOBI: size = b, idx ignored; contiguous blocks of b rows,
 *     the last one shorter, P = bldiag(K_y) (Sec. 3.3.1).
 *   KPCG_PREC_FITC: size = m, idx as for Nystrom; P = Q + diag(K - Q) + sigma^2 I
 *     (Sec. 3.1).  With D = diag(K - Q) + sigma^2 the inversion lemma gives
 *     P^-1 = D^-1/2 [I - K~ (K_UU + K~^T K~)^-1 K~^T] D^-1/2, K~ = D^-1/2 K_XU;
 *     K_UU and the inner matrix are factored with the same jitter rule.
 *   KPCG_PREC_NONE: removes the preconditioner.
 * In the mixed modes the preconditioner approximates the inner operator, so
 * it is built with noise sigma^2 (1 + inner_shift); it is rebuilt when the
 * mode or the shift changes.  Returns KPCG_ERR_NOT_SPD if a factorization
 * fails (the handle is then left without a preconditioner). */
kpcg_status kpcg_precond(kpcg_t h, int32_t kind, int64_t size, const int64_t* idx);

/* Build the random-feature preconditioner of Sec. 3.2 (KPCG_PREC_SPECTRAL).
 * K is approximated by K^_ij = (s^2/m) sum_r cos(2 pi s_r^T (x_i - x_j)) =
 * (Phi Phi^T)_ij, Phi_i = sqrt(s^2/m) [cos(2 pi s_r^T x_i), sin(2 pi s_r^T x_i)]_r
 * (n x 2m), with spectral points s_r ~ N(0, Lambda / (4 pi^2)), Lambda =
 * diag(1/l_r^2).  The random draws are an input: omega (host, m x d row-major,
 * float64) holds standard-normal values and s_r = omega_r / (2 pi l), so the
 * same draws serve every theta (the preconditioner is rebuilt from them after
 * kpcg_set_theta).  P^-1 = sigma^-2 [I - Phi (sigma^2 I + Phi^T Phi)^-1 Phi^T]
 * (the inversion lemma; the printed (I + Phi^T Phi) holds only for unit noise),
 * the inner 2m x 2m matrix factored with the jitter rule of kpcg_precond.
 * m in [1, 2048]; values must be finite.  In the mixed modes it is built for
 * the shifted inner noise, like the other kinds. */
kpcg_status kpcg_precond_spectral(kpcg_t h, int64_t m, const double* omega);

/* Build the PITC preconditioner of Sec. 3.1 (KPCG_PREC_PITC):
 * P = Q + bldiag(K - Q) + sigma^2 I, Q = K_XU K_UU^-1 K_UX on the m inducing
 * points idx (host, sorted, distinct, as for Nystrom), blocks of b contiguous
 * rows in input order (the last one shorter).  As the paper says, the block
 * diagonal D = bldiag(K - Q) + sigma^2 I takes the place of sigma^2 I in the
 * inversion lemma: with D = L_D L_D^T (block Cholesky, FP64) and
 * K~ = L_D^-1 K_XU, P^-1 = L_D^-T [I - K~ (K_UU + K~^T K~)^-1 K~^T] L_D^-1.
 * K_UU and the inner matrix use the jitter rule of kpcg_precond; a block of D
 * that does not factor returns KPCG_ERR_NOT_SPD.  m in [1, min(n, 4096)],
 * b in [1, 4096].  Set-up costs O(n m^2 + n b m); b = 1 is FITC. */
kpcg_status kpcg_precond_pitc(kpcg_t h, int64_t m, const int64_t* idx, int64_t b);

/* O = (K + sigma^2 I) V for c columns (device float64, column-major), the
 * matrix-free product of Sec. 2.1.  impl 0: entries and sums in native FP64;
 * impl 1: the double-float product of KPCG_DF64 and of the outer loop of the
 * mixed modes (FP32-pair arithmetic, about 44 bits per entry, sums carried as
 * FP32 pairs and added in FP64); for d <= 10 its squared distances come from
 * exact integer level sums of 8-bit slices of x' on the tensor cores, each
 * pair of points evaluated once for both triangles of K (n > 128), for
 * larger d from exact grid differences on the FP32 pipe;
 * impl 2: the sliced tensor-core kernel of KPCG_TCX_IR with V as FP32 pairs
 * (entries to FP32 accuracy, compensated sums, FP64 out; d <= 10);
 * impl 3: impl 1 with the FP32-pipe distances at every d;
 * impl 4: impl 1 evaluating every entry of K (no use of its symmetry;
 * d <= 10). */
kpcg_status kpcg_matvec_f64(kpcg_t h, const double* V, int64_t ldv, int32_t c, double* O,
                            int64_t ldo, int32_t impl);

/* O = (K + sigma^2 I) V in reduced precision (device float32).
 * impl 0: FP32 entries by direct differences on the CUDA cores;
 * impl 1: the tensor-core kernel KPCG_TC_IR iterates with (tcgen05 BF16x3
 *         split exponent, FP32 accumulate, exp2 and contraction in FP32);
 *         d <= 20, else KPCG_ERR_ARG.  A bounded wait that expires inside
 *         the kernel returns KPCG_ERR_TIMEOUT;
 * impl 2: the KPCG_FP32X_IR inner kernel (exact differences of the split
 *         inputs, compensated sums) with exp2 on the MUFU (ex2.approx);
 * impl 3: the same with a polynomial exp2 on the FMA pipe (the one the
 *         solver uses); impl 2 and 3 need d <= 16;
 * impl 4: the KPCG_TCX_IR inner kernel (tcgen05 on sliced per-point-exact
 *         operands, compensated row sums); d <= 10, a bounded wait that
 *         expires returns KPCG_ERR_TIMEOUT.
 * impl 5: tcgen05 for both contractions: the exponent as impl 1, then the
 *         exponentiated tile as FP16 (hi, lo) pairs in tensor memory against
 *         V as FP16 pairs scaled per column (~2^-21 relative per product);
 *         the KPCG_TC_IR inner product for blocks of 4 or more columns; d <= 20,
 *         KPCG_ERR_TIMEOUT as impl 1.
 * impl 6: the entries of impl 1 on symmetric tile pairs, one column at a
 *         time: each pair of 128-point tiles evaluated once for its row and
 *         its mirrored column sums (FP32, partials added in FP64); the
 *         KPCG_TC_IR inner product for blocks of up to 3 columns (n > 128;
 *         a single tile uses impl 1); d <= 20, KPCG_ERR_TIMEOUT as impl 1. */
kpcg_status kpcg_matvec_f32(kpcg_t h, const float* V, int64_t ldv, int32_t c, float* O,
                            int64_t ldo, int32_t impl);

/* Z = P^{-1} R with the preconditioner as built for the current mode
 * (device float64). */
kpcg_status kpcg_precond_apply_f64(kpcg_t h, const double* R, int64_t ldr, int32_t c, double* Z,
                                   int64_t ldz);

/* Solve (K + sigma^2 I) Xout = B for c columns (device float64), Algorithm 1
 * with the textbook recurrence, each column with its own scalars.  X0 is the
 * initial guess (device, ldx) or NULL for zero.  tol follows opt.tol_mode.
 * iters (host, nullable, c entries) receives per-column CG iterations.
 * Xout holds the best iterate also on KPCG_ERR_NO_CONVERGENCE.  A zero
 * column of B yields a zero solution in 0 iterations. */
kpcg_status kpcg_solve(kpcg_t h, const double* B, int64_t ldb, int32_t c, double tol,
                       const double* X0, double* Xout, int64_t ldx, int32_t* iters,
                       kpcg_info* info);

/* G_q = dK/dtheta_q W for q = log l_1..log l_d (ARD) or log l (isotropic),
 * then log s^2: the derivative products of Eq. 2 (device float64), entries
 * and sums in native FP64 (the trace term of the gradient cancels most of the
 * magnitude of these products).  G holds n_theta = (ard ? d : 1) + 1 blocks
 * of n x c, block q at G + q*ldg*c, column k at + k*ldg.  The noise
 * derivative sigma^2 W is left to the caller. */
kpcg_status kpcg_dkv(kpcg_t h, const double* W, int64_t ldw, int32_t c, double* G, int64_t ldg);

/* Stochastic gradient of log p(y|theta) (Eq. 2, trace by Rademacher probes as
 * in Sec. 2.1):  g_q = -1/2 (1/t) sum_k w_k^T dK_q r_k + 1/2 a^T dK_q a, with
 * [a, w_1..w_t] = K_y^{-1} [y, r_1..r_t] solved as one block to tol.
 * alpha0 (device, n doubles, nullable) is the initial iterate of the a column
 * (the probe columns start at zero).
 * y (device, n doubles), probes (device, n x t column-major, ld = n, entries
 * +-1, t >= 1).  grad (host) receives n_theta + 1 values:
 * d/dlog l_r (or d/dlog l), d/dlog s^2, d/dlog sigma^2.  alpha (device,
 * nullable) receives a = K_y^{-1} y.  The derivative products run in
 * double-float arithmetic (FP32 pairs, about 44 bits; native FP64 for d > 16):
 * the trace term cancels all but ~1e-5 of the magnitude of dK W, so FP32
 * entries would leave errors of ~3e-4 on the smaller gradient entries. */
kpcg_status kpcg_grad(kpcg_t h, const double* y, const double* probes, int32_t t, double tol,
                      const double* alpha0, double* grad, double* alpha, kpcg_info* info);

/* Predictions at ns test inputs (Sec. 2.1: the predictive mean and variance
 * need the kernel products of training and, for the variance, one linear
 * system per test point; Sec. 5 scores both).
 *   Xs: device float32, ns x d row-major (the layout of X); alpha: device, n,
 *   alpha = K_y^{-1} y (e.g. from kpcg_solve);
 *   mean (device, ns) = K(X_*, X) alpha, FP64 with entries rebuilt from X;
 *   var (device, ns, nullable) = the latent variance s^2 - k_*^T K_y^{-1} k_*
 *   with k_* = K(X, x_*): blocks of up to 16 test points are solved as
 *   right-hand sides with the handle's precision and preconditioner to tol.
 *   Add sigma^2 to var for the variance of a noisy target.
 * info (nullable) sums the variance solves.  ns = 0 is a no-op. */
kpcg_status kpcg_predict(kpcg_t h, const float* Xs, int64_t ns, const double* alpha,
                         double* mean, double* var, double tol, kpcg_info* info);

/* ---------------------------------------------------------------------------
 * GP classification with the probit likelihood p(y_i|f_i) = Phi(y_i f_i): the
 * Laplace approximation (Sec. 2.2; Appendix B, Algorithm "Laplace
 * approximation for GPs").  From f = 0, each Newton step computes
 * W = -d^2/df^2 log p(y|f) (diagonal) and g = d/df log p(y|f) at f,
 * b = W f + g, v = W^1/2 K b, solves B z = v with B = I + W^1/2 K W^1/2 by
 * PCG, and sets a = b - W^1/2 z, f = K a.  The loop stops when the objective
 * Psi(f) = log p(y|f) - 1/2 a^T f changes by at most newton_tol*max(1,|Psi|)
 * (the paper only says "until convergence").
 *   K: the handle's kernel (amplitude s^2, lengthscales); sigma^2 is unused.
 *   Products with K: the double-float kernel (KPCG_DF64's) for b, a and every
 *   certified residual; the per-point terms are FP64.  With the handle's
 *   precision KPCG_TC_IR or KPCG_FP32_IR each B-solve is the flexible-CG
 *   mixed solve of kpcg_solve (inner PCG on B in FP32 with the tensor-core or
 *   FP32 K.V, to opt.inner_tol; outer products and residuals double-float):
 *   B >= I, so reduced-precision products barely perturb it.  Otherwise PCG
 *   runs on the double-float B throughout.
 *   Preconditioner of B: with a Nystrom request on the handle (kpcg_precond,
 *   KPCG_PREC_NYSTROM) P_B = I + W^1/2 K_XU K_UU^-1 K_UX W^1/2 on the same
 *   inducing points, built at the first Newton step and rebuilt when W^1/2 has
 *   moved by more than 10% on some point since (a stale P_B is still SPD); with
 *   none, P_B = I; other kinds are rejected (KPCG_ERR_ARG).  From the second
 *   step on, each B-solve starts from the previous step's z.
 *   y: device, n labels, each +1 or -1 (checked).  f (device, n): the mode f^;
 *   a (device, n, nullable): a = K^-1 f^ (Appendix B), needed by predictions.
 *   newton_tol > 0, max_newton >= 1, cg_tol in (0, 1): each B-solve stops at
 *   ||v - B z|| <= cg_tol ||v|| (recomputed, at most 4 restarts).
 * Returns KPCG_ERR_NO_CONVERGENCE when max_newton steps end before the stop
 * test or a B-solve misses cg_tol (f and a then hold the last iterate). */
typedef struct {
    int32_t newton_steps;   /* Newton steps taken                                   */
    int32_t cg_iters_total; /* CG iterations over all B-solves                      */
    double psi;             /* Psi at the returned f                                */
    double max_rel_res;     /* worst recomputed ||v - B z|| / ||v|| of the B-solves */
    double time_ms;         /* wall time of the call on the host                    */
    double setup_ms;        /* part of time_ms spent building P_B                   */
    int32_t launches;       /* CUDA kernels this call launched                      */
    int32_t precond_builds; /* builds of P_B during the call                        */
} kpcg_laplace_info;

kpcg_status kpcg_laplace(kpcg_t h, const double* y, double newton_tol, int32_t max_newton,
                         double cg_tol, double* f, double* a, kpcg_laplace_info* info);

/* Predictions of the probit classifier at ns test inputs (Sec. 2.2; Appendix B,
 * "Prediction"), from the mode f and a = K^-1 f of kpcg_laplace on the same
 * handle and labels:
 *   mean (device, ns) = k_*^T a, the latent mean (FP64, entries rebuilt);
 *   var (device, ns, nullable) = s^2 - k_*^T W^1/2 B^-1 W^1/2 k_*, W and B at f:
 *   blocks of up to 16 test points are solved as right-hand sides of B by PCG to
 *   cg_tol (certified, preconditioned as in kpcg_laplace);
 *   prob (device, ns, nullable) = Phi(mean / sqrt(1 + var)), the predictive
 *   probability of y_* = +1 (the Gaussian integral of the probit likelihood).
 * Xs: device float32, ns x d row-major.  info (nullable): cg_iters_total sums
 * the blocks' iteration counts (the most any column took), max_rel_res is the
 * worst certified residual; newton_steps and psi are 0.  ns = 0 is a no-op. */
kpcg_status kpcg_laplace_predict(kpcg_t h, const double* y, const double* f, const double* a,
                                 const float* Xs, int64_t ns, double* mean, double* var,
                                 double* prob, double cg_tol, kpcg_laplace_info* info);

/* ---------------------------------------------------------------------------
 * Learned warm start.  Algorithm 1 takes an initial iterate x0; along a
 * hyperparameter trajectory a small network predicts coefficients c on a
 * basis B, and x0 = B c.  Two bases:
 *   - kernel basis: B = K(X, Z | theta) on m inducing points Z (kpcg_warm_basis);
 *   - snapshot basis: B = the q most recent solutions pushed along the
 *     trajectory, most recent first (kpcg_warm_snapshots, kpcg_warm_push).
 * The calls below fit and expand on the active basis (the last one chosen),
 * and provide the network (hand-written training and inference kernels).
 * ------------------------------------------------------------------------ */

/* Kernel basis Z = rows idx (host, m sorted distinct indices) of X.  ridge
 * (> 0) regularises the fit: c = argmin |K_XZ c - a|^2 + ridge c^T K_ZZ c.
 * Rebuilt for the current theta when needed (same pivot rule as Nystrom). */
kpcg_status kpcg_warm_basis(kpcg_t h, int64_t m, const int64_t* idx, double ridge);
/* Snapshot basis of depth q (1 .. 16), emptied.  ridge (> 0) regularises the
 * fit: c = argmin |S c - a|^2 + ridge (tr(S^T S) / q) |c|^2, with S the n x q
 * matrix of the stored solutions (FP64 Gram matrix, q x q Cholesky). */
kpcg_status kpcg_warm_snapshots(kpcg_t h, int32_t q, double ridge);
/* Store a solution (device, n doubles) as the newest snapshot; the oldest of q
 * is dropped.  Until q are stored, missing snapshots count as zero vectors. */
kpcg_status kpcg_warm_push(kpcg_t h, const double* a);
/* c (device, m or q doubles) = fitted coefficients of a (device, n doubles). */
kpcg_status kpcg_warm_fit(kpcg_t h, const double* a, double* c);
/* x0 (device, n doubles) = B c for c (device, m or q doubles). */
kpcg_status kpcg_warm_expand(kpcg_t h, const double* c, double* x0);

typedef struct kpcg_mlp* kpcg_mlp_t;

/* The network Linear(n_in,h1)-tanh-Linear(h1,h2)-tanh-Linear(h2,n_out).
 * params (host, float32) holds W1 (h1 x n_in, row-major), b1, W2 (h2 x h1), b2,
 * W3 (n_out x h2), b3 back to back.  Batches up to max_batch rows. */
kpcg_status kpcg_mlp_create(int32_t n_in, int32_t h1, int32_t h2, int32_t n_out,
                            const float* params, int32_t max_batch, void* stream,
                            kpcg_mlp_t* out);
/* out (device, batch x n_out) for inputs (device, batch x n_in, row-major);
 * bf16 != 0: BF16 weights and inputs, FP32 accumulation (inference). */
kpcg_status kpcg_mlp_forward(kpcg_mlp_t m, const float* inputs, int32_t batch, float* out,
                             int32_t bf16);
/* Gradient of the mean squared error w.r.t. params into grads (device, params
 * layout); loss (host, nullable). */
kpcg_status kpcg_mlp_grad(kpcg_mlp_t m, const float* inputs, const float* targets,
                          int32_t batch, float* grads, float* loss);
/* epochs full-batch Adam steps (beta 0.9, 0.999, eps 1e-8) at rate lr.  One
 * step is captured once as a CUDA graph for these pointers, batch and lr, and
 * replayed; the pointers must stay valid while the network is trained with
 * them.  loss (host, nullable) receives the loss before the last update. */
kpcg_status kpcg_mlp_train(kpcg_mlp_t m, const float* inputs, const float* targets,
                           int32_t batch, int32_t epochs, float lr, float* loss);
/* Copy the parameters to params (host, float32, create layout). */
kpcg_status kpcg_mlp_get_params(kpcg_mlp_t m, float* params);
void kpcg_mlp_destroy(kpcg_mlp_t m);
const char* kpcg_mlp_last_error(kpcg_mlp_t m);

/* The native-FP64 product O = (K + sigma^2 I) V of kpcg_matvec_f64 (impl 0)
 * for callers that cannot allocate device memory: for example a host program
 * whose GPU memory is entirely reserved by another allocator (a framework's
 * pool that has claimed the device), or a latency-critical caller that must
 * not pay cudaMalloc's implicit device synchronisation.  The paper has no
 * counterpart; it is a deployment variant of the product of Sec. 2.1.
 *   X: device float32 n x d row-major; log_theta: host, d+1 (ard) or 2 values
 *   as in kpcg_create; V, O: device float64, column-major, ldv/ldo >= n;
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * It allocates nothing: its scratch (column means, scaled inputs, split
 * partial sums) is one static device array of 16 MiB that every GPU loading
 * the library holds until exit.  Sizes needing more are rejected with
 * KPCG_ERR_ARG and a message; on a 152-SM GPU every n below 74 880 fits for
 * d <= 8 (131 064 for d <= 4, 43 680 for d <= 16, 24 960 for d <= 32); n above
 * 2^31 is rejected the same way.  X, V and O must be device (or managed)
 * pointers, X 4-byte and V, O 8-byte aligned (else KPCG_ERR_ARG).  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress)
 * while the device is current and keeps it for the life of the process; if
 * you capture streams, make that first call before a capture begins, and do
 * not call it again on a device after cudaDeviceReset (the kept address would
 * be stale).  Every call shares the array and leaves its contents behind, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  The call synchronises the stream before it returns.  On
 * error the message is available from kpcg_last_error(NULL). */
kpcg_status kpcg_matvec_f64_noalloc(const float* X, int64_t n, int32_t d,
                                    const double* log_theta, int32_t ard, double noise_var,
                                    const double* V, int64_t ldv, int32_t c, double* O,
                                    int64_t ldo, void* stream);

/* Measured issue rates of the pipes that bound the kernel products (Sec. 2.1
 * products rebuild K's entries, so they are limited by arithmetic, not by
 * memory): out (host, 7 doubles) receives
 *   [0] FP32 FMA lane-instructions per second,
 *   [1] MUFU ex2.approx.ftz.f32 lane-instructions per second,
 *   [2] FP64 FMA lane-instructions per second,
 *   [3..5] the SM clock in MHz seen inside each of the three probes (clock64
 *          cycles over %globaltimer nanoseconds on one CTA),
 *   [6] the number of SMs.
 * Each probe runs about 20 ms on the current device (stream: cudaStream_t,
 * NULL = legacy default), dependent chains of one instruction kind on every
 * SM.  The paper has no counterpart: this is a measurement tool for the
 * rooflines of the library's kernels.  On error the message is available
 * from kpcg_last_error(NULL). */
kpcg_status kpcg_probe_rates(void* stream, double* out);

/* ---- Many independent systems of uneven size, solved together ----------
 * Each problem is an independent system (K_p + sigma_p^2 I) x = b of Eq. 1
 * with its own inputs, hyperparameters and Nystrom preconditioner (Sec. 3.1);
 * every one of its c right-hand sides runs its own CG (Algorithm 1) and stops
 * on its own.  The solve is the mixed-precision one (KPCG_TC_IR): an FP64
 * flexible-CG outer loop (double-float direction products, native-FP64 residuals) around an
 * inner FP32 PCG whose products with K are ONE persistent tensor-core launch
 * over the tiles of all problems, and whose preconditioner applies are one
 * batched launch sequence.
 *
 * Block layout: every batch vector is a device float64 (or float32 for the
 * test entry points) column-major ld x (nprob * c) array, ld >= max_p n_p;
 * column p*c + k holds the k-th vector of problem p in rows 0 .. n_p-1.  Rows
 * n_p .. ld-1 of an input are ignored, of an output set to zero. */
typedef struct kpcg_batch* kpcg_batch_t;
typedef struct {
    const float* X;          /* device, n x d row-major, copied by create */
    int64_t n;
    int32_t d;               /* 1 .. 16 */
    int32_t ard;
    const double* log_theta; /* host, d+1 (ard) or 2 values as in kpcg_create */
    double noise_var;        /* sigma^2 > 0 */
    int64_t m;               /* Nystrom inducing points, 0 = no preconditioner */
    const int64_t* idx;      /* host, m sorted distinct row indices (NULL when m = 0) */
} kpcg_problem;

/* Copies every problem (one internal handle each; see kpcg_create and
 * kpcg_precond for their checks).  opt: NULL = defaults with precision
 * KPCG_TC_IR; any other precision is rejected.  stream: cudaStream_t. */
kpcg_status kpcg_batch_create(int32_t nprob, const kpcg_problem* probs,
                              const kpcg_options* opt, void* stream, kpcg_batch_t* out);
/* Solve every system for its c right-hand sides B (device, block layout) to
 * ||b - K_y x|| <= tol ||b|| per column, the residual recomputed in FP64
 * (the outer loop's direction products use the double-float kernel).  X: device,
 * block layout (caller-owned).  iters, rel_res (host, nprob*c, nullable):
 * inner PCG iterations and final relative residual per column.  Returns
 * KPCG_ERR_NO_CONVERGENCE (X holds the last iterate) if a column missed tol. */
kpcg_status kpcg_batch_solve(kpcg_batch_t b, const double* B, int64_t ld, int32_t c, double tol,
                             double* X, int32_t* iters, double* rel_res, kpcg_info* info);
/* The batched tensor-core product O = (K_p + sigma_p^2 (1 + inner_shift) I) V
 * for every problem (device float32, block layout): the inner operator of the
 * solve, exposed for tests and benchmarks. */
kpcg_status kpcg_batch_matvec_f32(kpcg_batch_t b, const float* V, int64_t ld, int32_t c,
                                  float* O);
/* The batched preconditioner apply Z = P_p^{-1} R (device float32, block
 * layout); problems without inducing points return Z = R. */
kpcg_status kpcg_batch_precond_apply_f32(kpcg_batch_t b, const float* R, int64_t ld, int32_t c,
                                         float* Z);
/* Autotuner of the batched product for c columns per problem: times each
 * candidate length of the work-list items (1 .. 64 column tiles of 128) with
 * each contraction path (see kpcg_batch_set_contraction) on one persistent
 * CTA per SM with CUDA events and keeps the fastest.  Runs by itself before
 * the first product unless kpcg_batch_set_tiling fixed the tiling.
 * Outputs (host, nullable): the chosen length, CTAs, and its time in ms. */
kpcg_status kpcg_batch_tune(kpcg_batch_t b, int32_t c, int32_t* tiles_per_item, int32_t* ctas,
                            float* best_ms);
/* The second contraction of the batched product (the exponentiated tile
 * times V): 0 FP32 FMAs in the epilogue, pairs of row tiles sharing each
 * shared-memory read of V; 1 the tile as FP16 (hi, lo) pairs in tensor memory
 * against V as FP16 pairs scaled per problem and column, on the tensor cores
 * (d <= 20; ~2^-21 relative per product); -1 (default) the autotuner's
 * choice, or with a fixed tiling the tensor cores from 4 columns per problem.
 * KPCG_ERR_ARG for another mode or mode 1 with a problem of d > 20. */
kpcg_status kpcg_batch_set_contraction(kpcg_batch_t b, int32_t mode);
/* Replace the options of the batch and of its problems (precision must stay
 * KPCG_TC_IR).  With opt->profile == 0 the inner CG replays chunks of
 * check_every iterations from a captured CUDA graph; with profiling on it
 * launches kernel by kernel so each kind can be timed. */
kpcg_status kpcg_batch_set_options(kpcg_batch_t b, const kpcg_options* opt);
/* Fix the tiling (ctas = 0: one CTA per SM); disables the autotuner. */
kpcg_status kpcg_batch_set_tiling(kpcg_batch_t b, int32_t tiles_per_item, int32_t ctas);
/* max_p n_p: the smallest valid ld. */
int64_t kpcg_batch_max_n(kpcg_batch_t b);
void kpcg_batch_destroy(kpcg_batch_t b);
/* Message of the last failing call on b (NULL: of the last failed create). */
const char* kpcg_batch_last_error(kpcg_batch_t b);

/* Release the handle and every device buffer it owns.  NULL is ignored. */
void kpcg_destroy(kpcg_t h);

/* Message of the last failing call on h (or of the last failed create when
 * h is NULL).  Valid until the next call on h. */
const char* kpcg_last_error(kpcg_t h);

#ifdef __cplusplus
}
#endif
#endif /* KPCG_H */
