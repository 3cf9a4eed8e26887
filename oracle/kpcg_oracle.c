/*
 * kpcg_oracle.c -- plain FP64 CPU oracle for preconditioned CG on kernel
 * matrices (Cutajar, Osborne, Cunningham, Filippone, "Preconditioning Kernel
 * Matrices", ICML 2016).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header or constant with the CUDA
 * path.  Everything is double precision, entries are built by direct
 * differences (never by the norm expansion), and loops follow the defining
 * formulas without blocking or reordering beyond an OpenMP split over rows.
 *
 * Notation: the kernel amplitude is s2 (the paper's sigma^2 in Eq. 1), the
 * noise variance is sigma2 (the paper's lambda, K_y = K + lambda I, Sec. 2.1),
 * lengthscales are ell[r] (the paper's l_r).
 *
 * Layouts: X is row-major n x d.  Block vectors (right-hand sides, iterates)
 * are column-major with a leading dimension.  Dense matrices are row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. 1: k(x_i, x_j) = s2 * exp(-1/2 sum_r (x_ir - x_jr)^2 / l_r^2). */
static double rbf(const double* xi, const double* xj, int d, const double* ell, double s2) {
    double a = 0.0;
    for (int r = 0; r < d; ++r) {
        double t = (xi[r] - xj[r]) / ell[r];
        a += t * t;
    }
    return s2 * exp(-0.5 * a);
}

/* Cross Gram matrix G[i*m + j] = k(X_i, Z_j)  (Eq. 1). */
void or_gram(const double* X, int64_t n, const double* Z, int64_t m, int d, const double* ell,
             double s2, double* G) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j) G[i * m + j] = rbf(X + i * d, Z + j * d, d, ell, s2);
}

/* Matrix-free O = (K + sigma2 I) V for a block of c columns (Sec. 2.1: the
 * only operation CG needs is a product with K_y).  Each entry K_ij is
 * recomputed from X; nothing n x n is stored. */
void or_kyv(const double* X, int64_t n, int d, const double* ell, double s2, double sigma2,
            const double* V, int64_t ldv, int c, double* O, int64_t ldo) {
#pragma omp parallel
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)(c > 0 ? c : 1));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            for (int k = 0; k < c; ++k) acc[k] = sigma2 * V[i + k * ldv];
            for (int64_t j = 0; j < n; ++j) {
                double kij = rbf(X + i * d, X + j * d, d, ell, s2);
                for (int k = 0; k < c; ++k) acc[k] += kij * V[j + k * ldv];
            }
            for (int k = 0; k < c; ++k) O[i + k * ldo] = acc[k];
        }
        free(acc);
    }
}

/* Derivative products for the gradient of Eq. 2 in log-parameters:
 *   dK_ij / d log l_r  = K_ij (x_ir - x_jr)^2 / l_r^2        (r < d)
 *   dK_ij / d log s2   = K_ij                                 (slot d)
 * G holds d+1 blocks, block q is n x c column-major with leading dim n:
 * G[q*n*c + i + k*n] = sum_j dK_ij/dtheta_q W[j + k*ldw].
 * The noise derivative sigma2*W is diagonal and left to the caller. */
void or_dkv(const double* X, int64_t n, int d, const double* ell, double s2, const double* W,
            int64_t ldw, int c, double* G) {
    const int64_t blk = n * (int64_t)c;
#pragma omp parallel
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)(d + 1) * (size_t)(c > 0 ? c : 1));
        double* sq = (double*)malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            memset(acc, 0, sizeof(double) * (size_t)(d + 1) * (size_t)c);
            for (int64_t j = 0; j < n; ++j) {
                const double* xi = X + i * d;
                const double* xj = X + j * d;
                double a = 0.0;
                for (int r = 0; r < d; ++r) {
                    double t = (xi[r] - xj[r]) / ell[r];
                    sq[r] = t * t;
                    a += sq[r];
                }
                double kij = s2 * exp(-0.5 * a);
                for (int k = 0; k < c; ++k) {
                    double w = W[j + k * ldw];
                    for (int r = 0; r < d; ++r) acc[r * c + k] += kij * sq[r] * w;
                    acc[d * c + k] += kij * w;
                }
            }
            for (int q = 0; q <= d; ++q)
                for (int k = 0; k < c; ++k) G[q * blk + i + k * n] = acc[q * c + k];
        }
        free(acc);
        free(sq);
    }
}

/* Textbook Cholesky (Golub & Van Loan, the reference the paper adapts PCG
 * from): A = L L^T, lower triangle of the row-major n x n matrix A is
 * overwritten by L, the strict upper triangle is zeroed.  Returns 0, or
 * j+1 when the j-th pivot is not positive. */
static int chol_thr(double* A, int64_t n, double thr) {
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > thr)) return (int)(j + 1);
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
    return 0;
}

int or_chol(double* A, int64_t n) { return chol_thr(A, n, 0.0); }

/* Solve L L^T x = b in place for c columns (column-major B, leading dim ldb). */
void or_chol_solve(const double* L, int64_t n, double* B, int64_t ldb, int c) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < c; ++k) {
        double* b = B + (int64_t)k * ldb;
        for (int64_t i = 0; i < n; ++i) {
            double t = b[i];
            for (int64_t q = 0; q < i; ++q) t -= L[i * n + q] * b[q];
            b[i] = t / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double t = b[i];
            for (int64_t q = i + 1; q < n; ++q) t -= L[q * n + i] * b[q];
            b[i] = t / L[i * n + i];
        }
    }
}

/* ---------------------------------------------------------------------
 * Nystrom preconditioner, Sec. 3.1.
 *   P = K_XU K_UU^{-1} K_UX + sigma2 I
 * Matrix inversion lemma applied to this P gives
 *   P^{-1} = sigma2^{-1} [ I - K_XU (sigma2 K_UU + K_UX K_XU)^{-1} K_UX ].
 * (The printed inverse omits the factor sigma2 on K_UU; it is only right for
 * sigma2 = 1.)  M = sigma2 K_UU + K_UX K_XU is SPD and is factored once.
 * The paper does not discuss the factorization of M.  With a small noise M
 * is nearly singular (condition numbers ~1e13 seen), where whether a
 * Cholesky factorization "succeeds" depends on rounding details.  The rule
 * here is deterministic: a factorization is accepted only if every pivot
 * exceeds NYS_PIVOT_TOL * max_k M_kk; otherwise jitter 1e-12 * tr(M)/m * 10^k,
 * k = 0..6, is added to the diagonal and the next level tried.
 * --------------------------------------------------------------------- */
#define NYS_PIVOT_TOL 3e-12

int or_nys_setup(const double* X, int64_t n, int d, const double* ell, double s2, double sigma2,
                 const int64_t* idx, int64_t m, double* KXU, double* M, double* jitter_out) {
    double* U = (double*)malloc(sizeof(double) * (size_t)(m * d));
    for (int64_t a = 0; a < m; ++a) memcpy(U + a * d, X + idx[a] * d, sizeof(double) * (size_t)d);
    or_gram(X, n, U, m, d, ell, s2, KXU);
    double* M0 = (double*)malloc(sizeof(double) * (size_t)(m * m));
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < m; ++a)
        for (int64_t b = 0; b < m; ++b) {
            double t = sigma2 * rbf(U + a * d, U + b * d, d, ell, s2);
            for (int64_t i = 0; i < n; ++i) t += KXU[i * m + a] * KXU[i * m + b];
            M0[a * m + b] = t;
        }
    double tr = 0.0, dmax = 0.0;
    for (int64_t a = 0; a < m; ++a) {
        tr += M0[a * m + a];
        if (M0[a * m + a] > dmax) dmax = M0[a * m + a];
    }
    int status = 1;
    double jit = 0.0;
    for (int k = -1; k <= 6 && status != 0; ++k) {
        jit = (k < 0) ? 0.0 : 1e-12 * tr / (double)m * pow(10.0, k);
        memcpy(M, M0, sizeof(double) * (size_t)(m * m));
        for (int64_t a = 0; a < m; ++a) M[a * m + a] += jit;
        status = chol_thr(M, m, NYS_PIVOT_TOL * dmax);
    }
    if (jitter_out) *jitter_out = jit;
    free(U);
    free(M0);
    return status;
}

/* Z = P^{-1} R with the factor L of M from or_nys_setup. */
void or_nys_apply(int64_t n, int64_t m, double sigma2, const double* KXU, const double* LM,
                  const double* R, int64_t ldr, int c, double* Z, int64_t ldz) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(m * c));
    for (int k = 0; k < c; ++k)
        for (int64_t a = 0; a < m; ++a) {
            double t = 0.0;
            for (int64_t i = 0; i < n; ++i) t += KXU[i * m + a] * R[i + k * ldr];
            w[a + k * m] = t;
        }
    or_chol_solve(LM, m, w, m, c);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < c; ++k) {
            double t = 0.0;
            for (int64_t a = 0; a < m; ++a) t += KXU[i * m + a] * w[a + k * m];
            Z[i + k * ldz] = (R[i + k * ldr] - t) / sigma2;
        }
    free(w);
}

/* ---------------------------------------------------------------------
 * Block-Jacobi preconditioner, Sec. 3.3.1: P = bldiag(K_y), contiguous
 * blocks of b rows in input order, the last block holding n mod b rows.
 * (The printed bldiag(K_y + lambda I) would count the noise twice, since
 * K_y already holds lambda I.)  Lbj stores the Cholesky factors of the
 * blocks one after another, block q at offset q*b*b (row-major bq x bq).
 * --------------------------------------------------------------------- */
int or_bj_setup(const double* X, int64_t n, int d, const double* ell, double s2, double sigma2,
                int64_t b, double* Lbj) {
    int64_t nb = (n + b - 1) / b;
    int status = 0;
    for (int64_t q = 0; q < nb; ++q) {
        int64_t r0 = q * b, bq = (n - r0 < b) ? (n - r0) : b;
        double* L = Lbj + q * b * b;
        or_gram(X + r0 * d, bq, X + r0 * d, bq, d, ell, s2, L);
        for (int64_t a = 0; a < bq; ++a) L[a * bq + a] += sigma2;
        int st = or_chol(L, bq);
        if (st && !status) status = (int)(r0 + st);
    }
    return status;
}

void or_bj_apply(int64_t n, int64_t b, const double* Lbj, const double* R, int64_t ldr, int c,
                 double* Z, int64_t ldz) {
    int64_t nb = (n + b - 1) / b;
    for (int k = 0; k < c; ++k)
        for (int64_t i = 0; i < n; ++i) Z[i + k * ldz] = R[i + k * ldr];
    for (int64_t q = 0; q < nb; ++q) {
        int64_t r0 = q * b, bq = (n - r0 < b) ? (n - r0) : b;
        or_chol_solve(Lbj + q * b * b, bq, Z + r0, ldz, c);
    }
}

/* ---------------------------------------------------------------------
 * Preconditioned CG, Algorithm 1 (adapted by the paper from Golub & Van
 * Loan), applied to each of the c columns independently.  The printed
 * algorithm has misprints; this follows the textbook recurrence:
 *   r0 = b - K_y x0, z0 = P^{-1} r0, p0 = z0, rho0 = r0^T z0
 *   q = K_y p;  alpha = rho / (p^T q);  x += alpha p;  r -= alpha q
 *   stop test;  z = P^{-1} r;  rho' = r^T z;  beta = rho'/rho;  p = z + beta p
 * Stop test: tol_mode 0 is ||r|| <= tol ||b|| (relative), tol_mode 1 is the
 * paper's absolute test ||r||^2 < n * tol (Sec. 4 uses tol = 1e-10).
 * When the recursive residual passes, the true residual b - K_y x is
 * recomputed; if it fails the test, CG restarts from x (at most 5 times).
 * p^T q <= 0 is a breakdown (K_y is SPD, so it can only come from rounding).
 *
 * kind: 0 none, 1 Nystrom (KXU, LM, m), 2 block-Jacobi (Lbj, b).
 * iters[k] receives the CG iterations of column k (-1 on breakdown),
 * relres[k] the recomputed ||b - K_y x|| / ||b||.  Returns 0 if every
 * column converged, 1 if some hit max_iter, 2 on a breakdown.
 * hist (nullable, max_iter + 1 entries) receives, for the first column, the
 * recursive ||r_i|| / ||b|| before each iteration i (entry 0: initial).
 * --------------------------------------------------------------------- */
typedef struct {
    int kind;
    int64_t n, m, b;
    double sigma2;
    const double *KXU, *LM, *Lbj;
} precond_t;

static void papply(const precond_t* P, const double* R, int64_t ldr, int c, double* Z, int64_t ldz) {
    if (P->kind == 1)
        or_nys_apply(P->n, P->m, P->sigma2, P->KXU, P->LM, R, ldr, c, Z, ldz);
    else if (P->kind == 2)
        or_bj_apply(P->n, P->b, P->Lbj, R, ldr, c, Z, ldz);
    else
        for (int k = 0; k < c; ++k)
            for (int64_t i = 0; i < P->n; ++i) Z[i + k * ldz] = R[i + k * ldr];
}

static double dotc(const double* a, const double* b, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

int or_pcg(const double* X, int64_t n, int d, const double* ell, double s2, double sigma2, int kind,
           const double* KXU, const double* LM, int64_t m, const double* Lbj, int64_t b,
           const double* B, int64_t ldb, int c, double tol, int tol_mode, int max_iter,
           const double* X0, double* Xout, int64_t ldx, int* iters, double* relres,
           double* hist) {
    precond_t P = {kind, n, m, b, sigma2, KXU, LM, Lbj};
    int rc = 0;
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    for (int k = 0; k < c; ++k) {
        const double* bk = B + (int64_t)k * ldb;
        double bnorm = sqrt(dotc(bk, bk, n));
        for (int64_t i = 0; i < n; ++i) x[i] = X0 ? X0[i + (int64_t)k * ldx] : 0.0;
        iters[k] = 0;
        if (bnorm == 0.0) {
            for (int64_t i = 0; i < n; ++i) Xout[i + (int64_t)k * ldx] = 0.0;
            relres[k] = 0.0;
            continue;
        }
        double thr2 = (tol_mode == 1) ? (double)n * tol : tol * tol * bnorm * bnorm;
        double* hk = (k == 0) ? hist : NULL;
        int restarts = 0, it = 0, done = 0, broke = 0;
        while (!done) {
            /* (re)start: r = b - K_y x */
            or_kyv(X, n, d, ell, s2, sigma2, x, n, 1, q, n);
            for (int64_t i = 0; i < n; ++i) r[i] = bk[i] - q[i];
            if (dotc(r, r, n) <= thr2) break;
            if (restarts > 5 || it >= max_iter) break;
            papply(&P, r, n, 1, z, n);
            for (int64_t i = 0; i < n; ++i) p[i] = z[i];
            double rho = dotc(r, z, n);
            if (hk) hk[it] = sqrt(dotc(r, r, n)) / bnorm;
            int conv = 0;
            while (it < max_iter) {
                or_kyv(X, n, d, ell, s2, sigma2, p, n, 1, q, n);
                double pq = dotc(p, q, n);
                ++it;
                if (!(pq > 0.0)) { broke = 1; break; }
                double alpha = rho / pq;
                for (int64_t i = 0; i < n; ++i) {
                    x[i] += alpha * p[i];
                    r[i] -= alpha * q[i];
                }
                double rr = dotc(r, r, n);
                if (hk) hk[it] = sqrt(rr) / bnorm;
                if (rr <= thr2) { conv = 1; break; }
                papply(&P, r, n, 1, z, n);
                double rho1 = dotc(r, z, n);
                double beta = rho1 / rho;
                rho = rho1;
                for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
            }
            if (broke || !conv) break;
            ++restarts; /* recursive residual passed: loop re-checks the true one */
        }
        or_kyv(X, n, d, ell, s2, sigma2, x, n, 1, q, n);
        double rr = 0.0;
        for (int64_t i = 0; i < n; ++i) rr += (bk[i] - q[i]) * (bk[i] - q[i]);
        relres[k] = sqrt(rr) / bnorm;
        for (int64_t i = 0; i < n; ++i) Xout[i + (int64_t)k * ldx] = x[i];
        iters[k] = broke ? -1 : it;
        if (broke) rc = 2;
        else if (rr > thr2 && rc == 0) rc = 1;
    }
    free(x); free(r); free(z); free(p); free(q);
    return rc;
}
