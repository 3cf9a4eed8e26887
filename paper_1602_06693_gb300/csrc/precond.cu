// Preconditioners of Sec. 3: Nystrom (Sec. 3.1) and block-Jacobi (Sec. 3.3.1).
//
// Nystrom.  P = K_XU K_UU^{-1} K_UX + sigma^2 I, inverted by the matrix
// inversion lemma as P^{-1} = sigma^{-2} [I - K_XU M^{-1} K_UX] with
// M = sigma^2 K_UU + K_UX K_XU (the printed inverse drops the sigma^2 on K_UU).
// K_XU holds FP64 entries as exact FP32 pairs; M is formed from it with FP64
// products and sums (see syrk_kxu_kernel for why nothing less will do).  M = L L^T is factored in FP64 and
// L^{-1} formed explicitly (stored as U = L^{-T}, row-major), so an apply is
// two skinny products with K_XU and two m x m triangular products.  K_UX r uses
// compensated FP32 (Dot2) on the pairs, the rest is FP64: with sigma^2 small
// the difference r - K_XU M^{-1} K_UX r cancels almost completely along the
// leading eigenvectors, and a plain FP32 accumulation there destroys the
// preconditioner.
//
// Block-Jacobi.  P = bldiag(K_y), contiguous blocks of b rows (the last one
// shorter).  Each block is factored in FP64 and its inverse factor stored;
// an apply is two triangular products per block, FP64 accumulation.
//
// Factorizations are blocked right-looking Cholesky (diagonal block on one
// CTA, panel solve and trailing update across the grid), batched over
// matrices of equal leading dimension.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "kpcg_internal.cuh"
#include "batch.cuh"
#include "precond.cuh"

namespace kpcg {

// Raise a kernel's dynamic shared-memory limit once per size (the first
// call runs outside any graph capture; later ones find it raised).
static void raise_smem_limit(const void* kern, size_t smem) {
    static std::map<const void*, size_t> done;
    size_t& have = done[kern];
    if (smem <= have) return;
    KPCG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    have = smem;
}

namespace {

constexpr int NB = 32;  // panel width of the blocked Cholesky

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Size of matrix q in a batch of blocks of a length-n_total index range.
__device__ __forceinline__ int64_t bsize(int64_t q, int64_t b, int64_t n_total) {
    const int64_t r0 = q * b;
    return (n_total - r0 < b) ? (n_total - r0) : b;
}

// Factor the nb x nb diagonal block at (j0, j0) of matrix q in place; a pivot
// not above thr fails the factorization.
__global__ void potrf_diag_kernel(double* A, int64_t stride, int64_t b, int64_t n_total,
                                  int64_t j0, int* status, double thr) {
    __shared__ double S[NB][NB + 1];
    __shared__ int bad;
    const int64_t q = blockIdx.x;
    const int64_t bq = bsize(q, b, n_total);
    if (j0 >= bq || status[q]) return;
    const int nb = (int)min((int64_t)NB, bq - j0);
    double* M = A + q * stride;
    const int64_t ld = bq;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e / nb, c = e % nb;
        S[r][c] = M[(j0 + r) * ld + j0 + c];
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double piv = S[j][j];
            if (!(piv > thr) || !isfinite(piv)) {
                bad = 1;
            } else {
                S[j][j] = sqrt(piv);
            }
        }
        __syncthreads();
        if (bad) {
            if (threadIdx.x == 0) status[q] = (int)(j0 + j + 1);
            return;
        }
        const double ljj = S[j][j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) S[i][j] /= ljj;
        __syncthreads();
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, k = e % nb;
            if (i > j && k > j && k <= i) S[i][k] -= S[i][j] * S[k][j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e / nb, c = e % nb;
        M[(j0 + r) * ld + j0 + c] = (c <= r) ? S[r][c] : 0.0;
    }
}

// Panel solve: rows i >= j0+nb of columns j0..j0+nb-1 become L21 = A21 L11^{-T}.
__global__ void trsm_panel_kernel(double* A, int64_t stride, int64_t b, int64_t n_total,
                                  int64_t j0, const int* status) {
    __shared__ double L[NB][NB + 1];
    const int64_t q = blockIdx.y;
    const int64_t bq = bsize(q, b, n_total);
    if (j0 >= bq || status[q]) return;
    const int nb = (int)min((int64_t)NB, bq - j0);
    double* M = A + q * stride;
    const int64_t ld = bq;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e / nb, c = e % nb;
        L[r][c] = M[(j0 + r) * ld + j0 + c];
    }
    __syncthreads();
    const int64_t i = j0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bq) return;
    double x[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) x[t] = (t < nb) ? M[i * ld + j0 + t] : 0.0;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        if (t < nb) {
            double s = x[t];
#pragma unroll
            for (int u = 0; u < NB; ++u)
                if (u < t) s -= x[u] * L[t][u];
            x[t] = s / L[t][t];
        }
    }
#pragma unroll
    for (int t = 0; t < NB; ++t)
        if (t < nb) M[i * ld + j0 + t] = x[t];
}

// Trailing update A22 -= L21 L21^T on the lower triangle; 32x32 output tiles.
__global__ void syrk_update_kernel(double* A, int64_t stride, int64_t b, int64_t n_total,
                                   int64_t j0, const int* status) {
    __shared__ double Li[32][NB + 1];
    __shared__ double Lk[32][NB + 1];
    const int64_t q = blockIdx.z;
    const int64_t bq = bsize(q, b, n_total);
    if (j0 >= bq || status[q]) return;
    const int nb = (int)min((int64_t)NB, bq - j0);
    const int64_t t0 = j0 + nb;
    const int64_t ti = blockIdx.y, tk = blockIdx.x;
    if (tk > ti) return;
    const int64_t i0 = t0 + ti * 32, k0 = t0 + tk * 32;
    if (i0 >= bq) return;
    double* M = A + q * stride;
    const int64_t ld = bq;
    for (int e = threadIdx.x; e < 32 * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        Li[r][c] = (i0 + r < bq && c < nb) ? M[(i0 + r) * ld + j0 + c] : 0.0;
        Lk[r][c] = (k0 + r < bq && c < nb) ? M[(k0 + r) * ld + j0 + c] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 each
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
            const int r = ty * 2 + a, cc = tx * 2 + c2;
            const int64_t i = i0 + r, k = k0 + cc;
            if (i < bq && k < bq && k <= i) {
                double s = 0.0;
#pragma unroll
                for (int u = 0; u < NB; ++u) s = fma(Li[r][u], Lk[cc][u], s);
                M[i * ld + k] -= s;
            }
        }
}

// U = L^{-T}: warp w solves L x = e_j for column j, writing x into row j of U.
__global__ void trinv_kernel(const double* Lb, double* Ub, int64_t stride, int64_t b,
                             int64_t n_total, int64_t nmat) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    // Flat column index over the batch: matrix q holds columns [q*b, q*b+bq).
    const int64_t q = gw / b, j = gw % b;
    if (q >= nmat) return;
    const int64_t bq = bsize(q, b, n_total);
    if (j >= bq) return;
    const double* L = Lb + q * stride;
    double* U = Ub + q * stride + j * bq;  // row j of U
    for (int64_t i = lane; i < j; i += 32) U[i] = 0.0;
    if (lane == 0) U[j] = 1.0 / L[j * bq + j];
    __syncwarp();
    for (int64_t i = j + 1; i < bq; ++i) {
        const double* Li = L + i * bq;
        double s = 0.0;
        for (int64_t k = j + lane; k < i; k += 32) s = fma(Li[k], U[k], s);
        s = warp_sum(s);
        if (lane == 0) U[i] = -s / Li[i];
        __syncwarp();
    }
}

// ---------------------------------------------------------------- Nystrom
__global__ void gather_rows_f32(const float* __restrict__ src, const int64_t* __restrict__ idx,
                                int64_t m, int dp, float* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * dp) return;
    const int64_t a = e / dp;
    dst[e] = src[idx[a] * dp + (e - a * dp)];
}
__global__ void gather_rows_f64(const double* __restrict__ src, const int64_t* __restrict__ idx,
                                int64_t m, int dp, double* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * dp) return;
    const int64_t a = e / dp;
    dst[e] = src[idx[a] * dp + (e - a * dp)];
}

// part[s][a][b] = sum over rows of split s of KXU[i][a] KXU[i][b], lower tiles,
// in FP64 (entries are exact FP32 pairs, hi + lo).  M = noise K_UU + K_UX K_XU
// is nearly singular (kappa ~ 1e11 at noise 1e-4) and the preconditioner it
// defines implicitly inverts K_UU, whose small eigenvalues are far below the
// 2^-48 relative error of a compensated-FP32 sum divided by the noise: such
// errors made the preconditioner indefinite and doubled the PCG iteration
// count.  FP64 products and sums keep it at the accuracy of a direct FP64
// construction.
constexpr int ST = 64;  // output tile
constexpr int SR = 16;  // rows per stage
__global__ void __launch_bounds__(256)
    syrk_kxu_kernel(const float2* __restrict__ KXU, int64_t n, int64_t m, int64_t rows_per_split,
                    double* __restrict__ part) {
    __shared__ double Aa[SR][ST];
    __shared__ double Ab[SR][ST];
    const int64_t ta = blockIdx.y, tb = blockIdx.x;
    if (tb > ta) return;
    const int64_t a0 = ta * ST, b0 = tb * ST;
    const int64_t r0 = (int64_t)blockIdx.z * rows_per_split;
    const int64_t r1 = min(n, r0 + rows_per_split);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 4 x 4 outputs each
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
    for (int64_t rs = r0; rs < r1; rs += SR) {
        __syncthreads();
        for (int e = threadIdx.x; e < SR * ST; e += 256) {
            const int r = e / ST, c = e % ST;
            const int64_t i = rs + r;
            float2 ka = (i < r1 && a0 + c < m) ? KXU[i * m + a0 + c] : make_float2(0.f, 0.f);
            float2 kb = (i < r1 && b0 + c < m) ? KXU[i * m + b0 + c] : make_float2(0.f, 0.f);
            Aa[r][c] = (double)ka.x + (double)ka.y;
            Ab[r][c] = (double)kb.x + (double)kb.y;
        }
        __syncthreads();
#pragma unroll 2
        for (int r = 0; r < SR; ++r) {
            double va[4], vb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) va[u] = Aa[r][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 4; ++v) vb[v] = Ab[r][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(va[u], vb[v], acc[u][v]);
        }
    }
    double* P = part + (int64_t)blockIdx.z * m * m;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t a = a0 + ty * 4 + u, bb = b0 + tx * 4 + v;
            if (a < m && bb < m && bb <= a) P[a * m + bb] = acc[u][v];
        }
}

// M[a][b] += sum_s part[s][a][b] (lower), then mirror to the upper triangle.
__global__ void syrk_reduce_kernel(const double* __restrict__ part, int nsplit, int64_t m,
                                   double* __restrict__ M) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int64_t a = e / m, b = e % m;
    if (b > a) return;
    double s = M[e];
    for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * m * m + e];
    M[e] = s;
    M[b * m + a] = s;
}

__global__ void add_diag_kernel(double* M, int64_t m, double v) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < m) M[a * m + a] += v;
}

// Compensated dot-product accumulation (Ogita, Rump and Oishi, "Accurate sum
// and dot product", 2005, algorithm Dot2): each product is split exactly into
// p + pi by an FMA (TwoProduct), p is added to the running sum s with Knuth's
// TwoSum, and all rounding errors are gathered in c.  s + c is as accurate as
// a dot product computed in twice the FP32 precision, at FP32-pipe speed.
struct Acc2 {
    float s, c;
};
__device__ __forceinline__ void dot2_add(Acc2& a, float x, float y) {
    const float p = x * y;
    const float pi = fmaf(x, y, -p);
    const float t = a.s + p;
    const float z = t - a.s;
    const float sg = (a.s - (t - z)) + (p - z);
    a.s = t;
    a.c += pi + sg;
}

// w_part[s][k][a] = sum_{i in split s} KXU[i][a] R[i][k]; K_XU and R enter as
// FP32 pairs, products are split exactly and accumulated with Dot2.
constexpr int PC = 4;  // columns per pass
template <typename T>
__global__ void __launch_bounds__(256)
    nys_proj_kernel(const float2* __restrict__ KXU, int64_t n, int64_t m, const T* __restrict__ R,
                    int64_t ldr, int ncols, int64_t rows_per_split, double* __restrict__ part,
                    int c_total) {
    __shared__ float2 sr[128][PC];  // r split into float hi + lo
    const int64_t a = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t r1 = min(n, r0 + rows_per_split);
    Acc2 acc[PC];
#pragma unroll
    for (int k = 0; k < PC; ++k) acc[k] = {0.f, 0.f};
    for (int64_t rs = r0; rs < r1; rs += 128) {
        __syncthreads();
        for (int e = threadIdx.x; e < 128 * PC; e += 256) {
            const int k = e / 128, r = e % 128;
            double v = (rs + r < r1 && k < ncols) ? (double)R[rs + r + (int64_t)k * ldr] : 0.0;
            const float hi = (float)v;
            sr[r][k] = make_float2(hi, (float)(v - (double)hi));
        }
        __syncthreads();
        const int rn = (int)min((int64_t)128, r1 - rs);
        if (a < m) {
            const float2* Kp = KXU + rs * m + a;
#pragma unroll 4
            for (int r = 0; r < rn; ++r) {
                const float2 kv = __ldg(Kp + (int64_t)r * m);
#pragma unroll
                for (int k = 0; k < PC; ++k) {
                    dot2_add(acc[k], kv.x, sr[r][k].x);
                    acc[k].c = fmaf(kv.x, sr[r][k].y, fmaf(kv.y, sr[r][k].x, acc[k].c));
                }
            }
        }
    }
    if (a < m)
        for (int k = 0; k < ncols; ++k)
            part[((int64_t)blockIdx.y * c_total + k) * m + a] = (double)acc[k].s + (double)acc[k].c;
}

__global__ void sum_splits_kernel(const double* __restrict__ part, int nsplit, int64_t len,
                                  double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * len + e];
    out[e] = s;
}

// y_k = L^{-1} w_k with U = L^{-T} row-major: y_i = sum_{j <= i} U[j][i] w_j.
// A CTA owns 32 consecutive i; its 32 warps stride over j (coalesced rows of
// U), and the 32 partial sums of each i are added in a fixed order.
__global__ void __launch_bounds__(1024)
    tri_lower_apply_kernel(const double* __restrict__ U, int64_t m, const double* __restrict__ w,
                           double* __restrict__ y) {
    __shared__ double part[32][33];
    const int k = blockIdx.y;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    const double* wk = w + (int64_t)k * m;
    double s = 0.0;
    if (i < m)
        for (int64_t j = g; j <= i; j += 32) s = fma(U[j * m + i], wk[j], s);
    part[g][lane] = s;
    __syncthreads();
    if (g == 0 && i < m) {
        double t = 0.0;
        for (int q = 0; q < 32; ++q) t += part[q][lane];
        y[(int64_t)k * m + i] = t;
    }
}

// u_k = L^{-T} y_k: u_j = sum_{i >= j} U[j][i] y_i (warp per j).
__global__ void tri_upper_apply_kernel(const double* __restrict__ U, int64_t m,
                                       const double* __restrict__ y, double* __restrict__ u) {
    const int k = blockIdx.y;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= m) return;
    const double* yk = y + (int64_t)k * m;
    const double* Uj = U + j * m;
    double s = 0.0;
    for (int64_t i = j + lane; i < m; i += 32) s = fma(Uj[i], yk[i], s);
    s = warp_sum(s);
    if (lane == 0) u[(int64_t)k * m + j] = s;
}

// Z = (R - K_XU u) / sigma^2, warp per row, FP64 accumulation.  With a
// badly conditioned M (kappa ~ 1e11 at noise 1e-4), u = M^{-1} K_UX r has
// components up to ~1e6 that cancel to O(1) in K_XU u; a compensated-FP32 sum
// (2^-48) left ~3e-6 relative noise there and weakened the preconditioner,
// FP64 (2^-53) matches the direct solve.
template <typename T>
__global__ void __launch_bounds__(256)
    nys_back_kernel(const float2* __restrict__ KXU, int64_t n, int64_t m,
                    const double* __restrict__ u, int c, const T* __restrict__ R, int64_t ldr,
                    T* __restrict__ Z, int64_t ldz, double inv_noise) {
    extern __shared__ double su[];  // m * c
    for (int64_t e = threadIdx.x; e < m * c; e += blockDim.x) su[e] = u[e];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const float2* Ki = KXU + i * m;
        for (int k = 0; k < c; ++k) {
            const double* uk = su + (int64_t)k * m;
            double acc = 0.0;
            for (int64_t a = lane; a < m; a += 32) {
                const float2 kv = __ldg(Ki + a);
                acc = fma((double)kv.x + (double)kv.y, uk[a], acc);
            }
            const double sm = warp_sum(acc);
            if (lane == 0)
                Z[i + (int64_t)k * ldz] = (T)(((double)R[i + (int64_t)k * ldr] - sm) * inv_noise);
        }
    }
}

// ---------------------------------------------------------- block-Jacobi
// Dense block of K_y: A_q[a][b] = s2 exp(-|x'_a - x'_b|^2) + noise [a == b].
__global__ void bj_fill_kernel(const double* __restrict__ xs, int64_t n, int dp, double c0,
                               double noise, int64_t b, double* __restrict__ A) {
    const int64_t q = blockIdx.y;
    const int64_t bq = bsize(q, b, n);
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= bq * bq) return;
    const int64_t r = e / bq, c = e % bq;
    const double* xr = xs + (q * b + r) * dp;
    const double* xc = xs + (q * b + c) * dp;
    double acc = c0;
    for (int t = 0; t < dp; ++t) {
        const double d = xr[t] - xc[t];
        acc = fma(-d, d, acc);
    }
    A[q * b * b + e] = exp(acc) + (r == c ? noise : 0.0);
}

// z_blk = L^{-T} L^{-1} r_blk for block q, column k (one CTA each).
template <typename T>
__global__ void bj_apply_kernel(const double* __restrict__ Ub, int64_t n, int64_t b,
                                const T* __restrict__ R, int64_t ldr, T* __restrict__ Z,
                                int64_t ldz) {
    extern __shared__ double sm[];  // 2 * b
    const int64_t q = blockIdx.x;
    const int k = blockIdx.y;
    const int64_t bq = bsize(q, b, n);
    const int64_t r0 = q * b;
    const double* U = Ub + q * b * b;
    double* rv = sm;
    double* yv = sm + b;
    for (int64_t i = threadIdx.x; i < bq; i += blockDim.x)
        rv[i] = (double)R[r0 + i + (int64_t)k * ldr];
    __syncthreads();
    for (int64_t i = threadIdx.x; i < bq; i += blockDim.x) {
        double s = 0.0;
        for (int64_t j = 0; j <= i; ++j) s = fma(U[j * bq + i], rv[j], s);
        yv[i] = s;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    for (int64_t j = threadIdx.x >> 5; j < bq; j += nw) {
        const double* Uj = U + j * bq;
        double s = 0.0;
        for (int64_t i = j + lane; i < bq; i += 32) s = fma(Uj[i], yv[i], s);
        s = warp_sum(s);
        if (lane == 0) Z[r0 + j + (int64_t)k * ldz] = (T)s;
    }
}

}  // namespace

// Blocked Cholesky of a batch of SPD matrices (in place, lower) and the
// explicit inverse factor U = L^{-T}.  Returns the first failing status.
static int factor_and_invert(double* A, double* U, int64_t b, int64_t n_total, int64_t nmat,
                             int* status_dev, cudaStream_t st, double thr = 0.0) {
    KPCG_CUDA(cudaMemsetAsync(status_dev, 0, sizeof(int) * nmat, st));
    for (int64_t j0 = 0; j0 < b; j0 += NB) {
        potrf_diag_kernel<<<(unsigned)nmat, 256, 0, st>>>(A, b * b, b, n_total, j0, status_dev,
                                                          thr);
        KPCG_LAUNCHED("potrf_diag_kernel");
        const int64_t rows = b - j0 - NB;
        if (rows > 0) {
            dim3 g1((unsigned)((rows + 127) / 128), (unsigned)nmat);
            trsm_panel_kernel<<<g1, 128, 0, st>>>(A, b * b, b, n_total, j0, status_dev);
            KPCG_LAUNCHED("trsm_panel_kernel");
            const unsigned nt = (unsigned)((rows + 31) / 32);
            dim3 g2(nt, nt, (unsigned)nmat);
            syrk_update_kernel<<<g2, 256, 0, st>>>(A, b * b, b, n_total, j0, status_dev);
            KPCG_LAUNCHED("syrk_update_kernel");
        }
    }
    std::vector<int> hs((size_t)nmat);
    KPCG_CUDA(cudaMemcpyAsync(hs.data(), status_dev, sizeof(int) * nmat, cudaMemcpyDeviceToHost,
                              st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    for (int64_t q = 0; q < nmat; ++q)
        if (hs[(size_t)q]) return hs[(size_t)q] + (int)(q * b);
    const int64_t warps = nmat * b;
    trinv_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(A, U, b * b, b, n_total,
                                                                      nmat);
    KPCG_LAUNCHED("trinv_kernel");
    return 0;
}

// Inducing rows and K_XU (FP64 entries, direct differences, stored as exact
// FP32 pairs: at small noise the preconditioner needs FP64-accurate entries;
// an FP32 rounding of K_XU alone raised the PCG iteration count by 10-50%).
static void nys_gather_kxu(PrecondState& P, const float* xs32, const double* xs64, int64_t n,
                           int dp, double c0_64, const int64_t* idx_host, int64_t m,
                           cudaStream_t st) {
    P.n = n;
    P.m = m;
    int64_t* idx = P.idx.need((size_t)m);
    KPCG_CUDA(cudaMemcpyAsync(idx, idx_host, sizeof(int64_t) * m, cudaMemcpyHostToDevice, st));
    float* us32 = P.us32.need((size_t)m * dp);
    double* us64 = P.us64.need((size_t)m * dp);
    const unsigned g = (unsigned)((m * dp + 255) / 256);
    gather_rows_f32<<<g, 256, 0, st>>>(xs32, idx, m, dp, us32);
    KPCG_LAUNCHED("gather_rows_f32");
    gather_rows_f64<<<g, 256, 0, st>>>(xs64, idx, m, dp, us64);
    KPCG_LAUNCHED("gather_rows_f64");
    float2* KXU = P.KXU.need((size_t)n * m);
    kxu_pair_f64(xs64, n, us64, m, dp, c0_64, KXU, st);
}

// Factor A (m x m, from A0 plus jitter) into P.M = L and P.U = L^{-T} with the
// deterministic acceptance rule (the paper is silent): every pivot must exceed
// 3e-12 * max diag(A0), else the jitter 1e-12 tr(A0)/m 10^k, k = 0..6, is added;
// a nearly singular matrix otherwise "factors" or not depending on rounding,
// and pivots near zero make a useless preconditioner.  Returns the jitter.
static double factor_with_rule(PrecondState& P, const double* A0, int64_t m, cudaStream_t st,
                               const char* what) {
    std::vector<double> diag((size_t)m);
    KPCG_CUDA(cudaMemcpy2DAsync(diag.data(), sizeof(double), A0, sizeof(double) * (m + 1),
                                sizeof(double), (size_t)m, cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    double tr = 0.0, dmax = 0.0;
    for (double v : diag) {
        tr += v;
        dmax = std::max(dmax, v);
    }
    const double kPivotTol = 3e-12;
    double* M = P.M.need((size_t)m * m);
    double* U = P.U.need((size_t)m * m);
    int* status = P.status.need(1);
    int rc = 1;
    double jitter = 0.0;
    for (int k = -1; k <= 6 && rc; ++k) {
        jitter = (k < 0) ? 0.0 : 1e-12 * tr / (double)m * std::pow(10.0, (double)k);
        KPCG_CUDA(cudaMemcpyAsync(M, A0, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
        if (jitter > 0.0) {
            add_diag_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(M, m, jitter);
            KPCG_LAUNCHED("add_diag_kernel");
        }
        rc = factor_and_invert(M, U, m, m, 1, status, st, kPivotTol * dmax);
    }
    if (rc) fail(KPCG_ERR_NOT_SPD, std::string(what) + " is not positive definite after jitter");
    return jitter;
}

// M0 += K_UX K_XU (FP64 SYRK over the pairs of P.KXU, n x m), then M0 is
// factored by the rule.
static void nys_syrk_factor(PrecondState& P, int64_t n, int64_t m, cudaStream_t st,
                            const char* what) {
    double* M0 = P.M0.p;
    const int64_t tiles = (m + ST - 1) / ST;
    // row splits: one per 4096 rows (at most 64), and enough for about four
    // CTAs per SM over the lower tiles when m is small, with >= 4 SR rows each
    const int64_t lower = tiles * (tiles + 1) / 2;
    int64_t ns = std::max<int64_t>(std::min<int64_t>(64, (n + 4095) / 4096),
                                   (152 * 4 + lower - 1) / lower);
    ns = std::min<int64_t>(ns, std::max<int64_t>(1, n / (4 * SR)));
    int nsplit = (int)std::max<int64_t>(1, ns);
    const int64_t rps = ((n + nsplit - 1) / nsplit + SR - 1) / SR * SR;
    nsplit = (int)((n + rps - 1) / rps);
    double* part = P.scratch.need((size_t)nsplit * m * m);
    dim3 gs((unsigned)tiles, (unsigned)tiles, (unsigned)nsplit);
    syrk_kxu_kernel<<<gs, 256, 0, st>>>(P.KXU.p, n, m, rps, part);
    KPCG_LAUNCHED("syrk_kxu_kernel");
    syrk_reduce_kernel<<<(unsigned)((m * m + 255) / 256), 256, 0, st>>>(part, nsplit, m, M0);
    KPCG_LAUNCHED("syrk_reduce_kernel");
    P.jitter = factor_with_rule(P, M0, m, st, what);
}

// M0 = noise K_UU + K_UX K_XU, factored by the rule.
static void nys_inner(PrecondState& P, int64_t n, int64_t m, int dp, double c0_64, double noise,
                      cudaStream_t st) {
    double* M0 = P.M0.need((size_t)m * m);
    kuu_f64(P.us64.p, m, dp, c0_64, noise, 0.0, M0, st);
    nys_syrk_factor(P, n, m, st, "Nystrom inner matrix");
}

void nystrom_setup(PrecondState& P, const float* xs32, const double* xs64, int64_t n, int dp,
                   float c0_32, double c0_64, double noise, const int64_t* idx_host, int64_t m,
                   cudaStream_t st) {
    (void)c0_32;
    P.kind = KPCG_PREC_NYSTROM;
    P.noise = noise;
    P.apply_noise = noise;
    nys_gather_kxu(P, xs32, xs64, n, dp, c0_64, idx_host, m, st);
    nys_inner(P, n, m, dp, c0_64, noise, st);
    P.ready = true;
}

namespace {

// dq[i] = |L^{-1} k_i|^2 = k_i^T K_UU^{-1} k_i with U = L^{-T} row-major:
// (L^{-1} k)_a = sum_{b <= a} U[b][a] k_b.  One CTA per row, FP64.
__global__ void fitc_diag_kernel(const float2* __restrict__ KXU, int64_t n, int64_t m,
                                 const double* __restrict__ U, double* __restrict__ dq) {
    extern __shared__ double sk[];
    __shared__ double red[8];
    const int64_t i = blockIdx.x;
    for (int64_t a = threadIdx.x; a < m; a += blockDim.x) {
        const float2 kv = KXU[i * m + a];
        sk[a] = (double)kv.x + (double)kv.y;
    }
    __syncthreads();
    double s = 0.0;
    for (int64_t a = threadIdx.x; a < m; a += blockDim.x) {
        double v = 0.0;
        for (int64_t b = 0; b <= a; ++b) v = fma(U[b * m + a], sk[b], v);
        s = fma(v, v, s);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        dq[i] = t;
    }
}

// D_i = s2 + noise - dq_i (at least noise: diag(K - Q) >= 0), dscale_i = D_i^{-1/2},
// and row i of K_XU scaled by dscale_i (re-split into an exact FP32 pair).
__global__ void fitc_scale_kernel(float2* __restrict__ KXU, int64_t n, int64_t m,
                                  const double* __restrict__ dq, double s2, double noise,
                                  double* __restrict__ dscale) {
    const int64_t i = blockIdx.x;
    const double D = fmax(s2 + noise - dq[i], noise);
    const double sc = 1.0 / sqrt(D);
    if (threadIdx.x == 0) dscale[i] = sc;
    for (int64_t a = threadIdx.x; a < m; a += blockDim.x) {
        const float2 kv = KXU[i * m + a];
        const double v = ((double)kv.x + (double)kv.y) * sc;
        const float hi = (float)v;
        KXU[i * m + a] = make_float2(hi, (float)(v - (double)hi));
    }
}

}  // namespace

void fitc_setup(PrecondState& P, const float* xs32, const double* xs64, int64_t n, int dp,
                float c0_32, double c0_64, double s2, double noise, const int64_t* idx_host,
                int64_t m, cudaStream_t st) {
    (void)c0_32;
    P.kind = KPCG_PREC_FITC;
    P.noise = noise;
    P.apply_noise = 1.0;
    nys_gather_kxu(P, xs32, xs64, n, dp, c0_64, idx_host, m, st);
    // K_UU and its factor (the same acceptance rule), then diag(Q)
    double* Kuu = P.M0.need((size_t)m * m);
    kuu_f64(P.us64.p, m, dp, c0_64, 1.0, 0.0, Kuu, st);
    (void)factor_with_rule(P, Kuu, m, st, "K_UU");
    double* dq = P.w.need((size_t)n);
    fitc_diag_kernel<<<(unsigned)n, 256, sizeof(double) * (size_t)m, st>>>(P.KXU.p, n, m, P.U.p,
                                                                           dq);
    KPCG_LAUNCHED("fitc_diag_kernel");
    double* dsc = P.dscale.need((size_t)n);
    fitc_scale_kernel<<<(unsigned)n, 256, 0, st>>>(P.KXU.p, n, m, dq, s2, noise, dsc);
    KPCG_LAUNCHED("fitc_scale_kernel");
    // inner matrix K_UU + K~^T K~ (unit noise) and its factor
    nys_inner(P, n, m, dp, c0_64, 1.0, st);
    P.ready = true;
}

namespace {

// Row i of Phi: amp [cos(w_r . x~_i) | sin(w_r . x~_i)], r = 0..m-1 (cosines in
// columns 0..m-1, sines in m..2m-1), FP64 phases and values stored as exact
// FP32 pairs.  With x~ = (x - mu) / l, w_r . x~_i = 2 pi s_r . x_i - 2 pi s_r . mu
// for s_r = w_r / (2 pi l): the constant phase cancels in Phi Phi^T.  xs holds
// x~ sqrt(1/2) (the FP64 kernels' scaling), so om carries w sqrt(2).  One
// thread per (i, r).
__global__ void rff_kernel(const double* __restrict__ xs, int64_t n, int dp,
                           const double* __restrict__ om, int64_t m, double amp,
                           float2* __restrict__ Phi) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const int64_t i = e / m, r = e - i * m;
    double ph = 0.0;
    for (int k = 0; k < dp; ++k) ph = fma(om[r * dp + k], xs[i * dp + k], ph);
    double sn, cs;
    sincos(ph, &sn, &cs);
    cs *= amp;
    sn *= amp;
    const float ch = (float)cs, sh = (float)sn;
    Phi[i * 2 * m + r] = make_float2(ch, (float)(cs - (double)ch));
    Phi[i * 2 * m + m + r] = make_float2(sh, (float)(sn - (double)sh));
}

// dst[i][a] = sc[i] src[i][a] for n x m pairs, re-split into exact FP32 pairs.
__global__ void scale_pairs_kernel(const float2* __restrict__ src, int64_t n, int64_t m,
                                   const double* __restrict__ sc, float2* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const float2 kv = src[e];
    const double v = ((double)kv.x + (double)kv.y) * sc[e / m];
    const float hi = (float)v;
    dst[e] = make_float2(hi, (float)(v - (double)hi));
}

}  // namespace

void spectral_setup(PrecondState& P, const double* xs64, int64_t n, int dp, double s2,
                    double noise, const double* omega_host, int d, int64_t m, cudaStream_t st) {
    P.kind = KPCG_PREC_SPECTRAL;
    P.n = n;
    P.m = 2 * m;
    P.noise = noise;
    P.apply_noise = noise;
    std::vector<double> om((size_t)m * dp, 0.0);
    for (int64_t r = 0; r < m; ++r)
        for (int k = 0; k < d; ++k)
            om[(size_t)(r * dp + k)] = omega_host[r * d + k] * 1.4142135623730950488;
    double* omd = P.us64.need((size_t)m * dp);
    KPCG_CUDA(cudaMemcpyAsync(omd, om.data(), sizeof(double) * om.size(), cudaMemcpyHostToDevice,
                              st));
    float2* Phi = P.KXU.need((size_t)n * 2 * m);
    rff_kernel<<<(unsigned)((n * m + 255) / 256), 256, 0, st>>>(xs64, n, dp, omd, m,
                                                                std::sqrt(s2 / (double)m), Phi);
    KPCG_LAUNCHED("rff_kernel");
    // inner matrix noise I + Phi^T Phi
    const int64_t q = 2 * m;
    double* M0 = P.M0.need((size_t)q * q);
    KPCG_CUDA(cudaMemsetAsync(M0, 0, sizeof(double) * q * q, st));
    add_diag_kernel<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(M0, q, noise);
    KPCG_LAUNCHED("add_diag_kernel");
    nys_syrk_factor(P, n, q, st, "random-feature inner matrix");
    P.ready = true;
}

void laplace_precond_setup(PrecondState& P, DevBuf<float2>& kxu0, bool first, const float* xs32,
                           const double* xs64, int64_t n, int dp, double c0_64,
                           const double* sW, const int64_t* idx_host, int64_t m,
                           cudaStream_t st) {
    if (first || !kxu0.p) {
        nys_gather_kxu(P, xs32, xs64, n, dp, c0_64, idx_host, m, st);
        float2* k0 = kxu0.need((size_t)n * m);
        KPCG_CUDA(cudaMemcpyAsync(k0, P.KXU.p, sizeof(float2) * n * m, cudaMemcpyDeviceToDevice,
                                  st));
    }
    P.kind = KPCG_PREC_NYSTROM;
    P.n = n;
    P.m = m;
    P.noise = 1.0;
    P.apply_noise = 1.0;
    scale_pairs_kernel<<<(unsigned)((n * m + 255) / 256), 256, 0, st>>>(kxu0.p, n, m, sW,
                                                                        P.KXU.p);
    KPCG_LAUNCHED("scale_pairs_kernel");
    nys_inner(P, n, m, dp, c0_64, 1.0, st);
    P.ready = true;
}

namespace {

// V[i][a] = (L^{-1} k_i)_a = sum_{b <= a} U[b][a] k_ib, U = L^{-T} of K_UU
// (row-major); one CTA per row, FP64.
__global__ void pitc_v_kernel(const float2* __restrict__ KXU, int64_t n, int64_t m,
                              const double* __restrict__ U, double* __restrict__ V) {
    extern __shared__ double sk[];
    const int64_t i = blockIdx.x;
    for (int64_t a = threadIdx.x; a < m; a += blockDim.x) {
        const float2 kv = KXU[i * m + a];
        sk[a] = (double)kv.x + (double)kv.y;
    }
    __syncthreads();
    for (int64_t a = threadIdx.x; a < m; a += blockDim.x) {
        double v = 0.0;
        for (int64_t b = 0; b <= a; ++b) v = fma(U[b * m + a], sk[b], v);
        V[i * m + a] = v;
    }
}

// Block q of D = bldiag(K - Q) + noise I (row-major with its own size bq, the
// block-Jacobi layout): entry (r, c) = K(x_r, x_c) - v_r . v_c + noise [r = c],
// FP64, K from direct differences.  16 x 16 output tiles, V staged 32 columns
// at a time.
__global__ void __launch_bounds__(256)
    pitc_fill_kernel(const double* __restrict__ xs, int64_t n, int dp, double c0, double noise,
                     const double* __restrict__ V, int64_t m, int64_t b, double* __restrict__ A) {
    __shared__ double Vr[16][33];
    __shared__ double Vc[16][33];
    // blockIdx.x = (q * tiles + tile row) * tiles + tile column
    const int64_t tiles = (b + 15) / 16;
    const int64_t q = (int64_t)blockIdx.x / (tiles * tiles);
    const int64_t tt = (int64_t)blockIdx.x - q * tiles * tiles;
    const int64_t bq = bsize(q, b, n);
    const int64_t r0 = (tt / tiles) * 16, k0 = (tt % tiles) * 16;
    if (r0 >= bq || k0 >= bq) return;  // uniform over the CTA
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t base = q * b;
    double acc = 0.0;
    for (int64_t a0 = 0; a0 < m; a0 += 32) {
        for (int e = threadIdx.x; e < 16 * 32; e += 256) {
            const int rr = e >> 5, aa = e & 31;
            const int64_t a = a0 + aa;
            Vr[rr][aa] = (r0 + rr < bq && a < m) ? V[(base + r0 + rr) * m + a] : 0.0;
            Vc[rr][aa] = (k0 + rr < bq && a < m) ? V[(base + k0 + rr) * m + a] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int u = 0; u < 32; ++u) acc = fma(Vr[ty][u], Vc[tx][u], acc);
        __syncthreads();
    }
    const int64_t r = r0 + ty, c = k0 + tx;
    if (r < bq && c < bq) {
        const double* xr = xs + (base + r) * dp;
        const double* xc = xs + (base + c) * dp;
        double e = c0;
        for (int t = 0; t < dp; ++t) {
            const double d = xr[t] - xc[t];
            e = fma(-d, d, e);
        }
        A[q * b * b + r * bq + c] = exp(e) - acc + (r == c ? noise : 0.0);
    }
}

// Y = L_D^{-1} K_XU block by block: Y[i][a] = sum_{j <= i in i's block}
// U_D[j][i] K_XU[j][a] (U_D = L_D^{-T} per block, row-major), written as exact
// FP32 pairs.  Threads run along a (coalesced); blockIdx.x is the row i.
__global__ void pitc_y_kernel(const float2* __restrict__ KXU, int64_t n, int64_t m,
                              const double* __restrict__ UD, int64_t b,
                              float2* __restrict__ Y) {
    const int64_t i = blockIdx.x;
    const int64_t a = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (a >= m) return;
    const int64_t q = i / b;
    const int64_t bq = bsize(q, b, n);
    const int64_t r0 = q * b, ii = i - r0;
    const double* U = UD + q * b * b;
    double acc = 0.0;
    for (int64_t j = 0; j <= ii; ++j) {
        const float2 kv = KXU[(r0 + j) * m + a];
        acc = fma(U[j * bq + ii], (double)kv.x + (double)kv.y, acc);
    }
    const float hi = (float)acc;
    Y[i * m + a] = make_float2(hi, (float)(acc - (double)hi));
}

}  // namespace

void pitc_setup(PrecondState& P, const float* xs32, const double* xs64, int64_t n, int dp,
                double c0_64, double noise, const int64_t* idx_host, int64_t m, int64_t b,
                cudaStream_t st) {
    P.kind = KPCG_PREC_PITC;
    P.noise = noise;
    P.apply_noise = 1.0;
    P.b = b;
    nys_gather_kxu(P, xs32, xs64, n, dp, c0_64, idx_host, m, st);
    // K_UU = L L^T (the jitter rule), V = L^{-1} K_UX, Q = V^T V
    double* Kuu = P.M0.need((size_t)m * m);
    kuu_f64(P.us64.p, m, dp, c0_64, 1.0, 0.0, Kuu, st);
    (void)factor_with_rule(P, Kuu, m, st, "K_UU");
    double* V = P.tmp64.need((size_t)n * m);
    const size_t smem = sizeof(double) * (size_t)m;
    if (smem > 48 * 1024) raise_smem_limit((const void*)pitc_v_kernel, smem);
    pitc_v_kernel<<<(unsigned)n, 256, smem, st>>>(P.KXU.p, n, m, P.U.p, V);
    KPCG_LAUNCHED("pitc_v_kernel");
    // D = bldiag(K - Q) + noise I and its block factors L_D, U_D = L_D^{-T}
    const int64_t nb = (n + b - 1) / b;
    double* A = P.dblk.need((size_t)nb * b * b);
    double* UD = P.dinv.need((size_t)nb * b * b);
    const int64_t tiles = (b + 15) / 16;
    pitc_fill_kernel<<<(unsigned)(nb * tiles * tiles), 256, 0, st>>>(xs64, n, dp, c0_64, noise,
                                                                     V, m, b, A);
    KPCG_LAUNCHED("pitc_fill_kernel");
    int* status = P.status.need((size_t)std::max<int64_t>(nb, 1));
    const int rc = factor_and_invert(A, UD, b, n, nb, status, st);
    if (rc)
        fail(KPCG_ERR_NOT_SPD,
             "PITC diagonal block not positive definite near row " + std::to_string(rc - 1));
    // K~ = L_D^{-1} K_XU as pairs; it replaces K_XU for the inner matrix and the apply
    DevBuf<float2> Y;
    Y.need((size_t)n * m);
    pitc_y_kernel<<<dim3((unsigned)n, (unsigned)((m + 255) / 256)), 256, 0, st>>>(P.KXU.p, n, m, UD,
                                                                                  b, Y.p);
    KPCG_LAUNCHED("pitc_y_kernel");
    KPCG_CUDA(cudaStreamSynchronize(st));
    std::swap(P.KXU.p, Y.p);
    std::swap(P.KXU.count, Y.count);
    // inner matrix K_UU + K~^T K~ (unit noise) and its factor
    nys_inner(P, n, m, dp, c0_64, 1.0, st);
    P.ready = true;
}

void block_jacobi_setup(PrecondState& P, const double* xs64, int64_t n, int dp, double c0_64,
                        double noise, int64_t b, cudaStream_t st) {
    P.kind = KPCG_PREC_BLOCK_JACOBI;
    P.n = n;
    P.b = b;
    P.noise = noise;
    const int64_t nb = (n + b - 1) / b;
    double* A = P.M.need((size_t)nb * b * b);
    double* U = P.U.need((size_t)nb * b * b);
    dim3 g((unsigned)((b * b + 255) / 256), (unsigned)nb);
    bj_fill_kernel<<<g, 256, 0, st>>>(xs64, n, dp, c0_64, noise, b, A);
    KPCG_LAUNCHED("bj_fill_kernel");
    int* status = P.status.need((size_t)nb);
    const int rc = factor_and_invert(A, U, b, n, nb, status, st);
    if (rc)
        fail(KPCG_ERR_NOT_SPD,
             "block of K_y not positive definite near row " + std::to_string(rc - 1));
    P.ready = true;
}

template <typename T>
static void nystrom_apply(const PrecondState& P, const T* R, int64_t ldr, int c, T* Z,
                          int64_t ldz, cudaStream_t st) {
    const int64_t n = P.n, m = P.m;
    const int64_t ablk = (m + 255) / 256;
    int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((152 * 4 + ablk - 1) / ablk,
                                                             (n + 127) / 128));
    const int64_t rps = (n + nsplit - 1) / nsplit;
    nsplit = (int)((n + rps - 1) / rps);
    double* part = const_cast<PrecondState&>(P).wpart.need((size_t)nsplit * c * m);
    double* w = const_cast<PrecondState&>(P).w.need((size_t)c * m);
    double* y = const_cast<PrecondState&>(P).y.need((size_t)c * m);
    for (int k0 = 0; k0 < c; k0 += PC) {
        const int nc = std::min(PC, c - k0);
        dim3 g((unsigned)((m + 255) / 256), (unsigned)nsplit);
        nys_proj_kernel<T><<<g, 256, 0, st>>>(P.KXU.p, n, m, R + (int64_t)k0 * ldr, ldr, nc, rps,
                                              part + (int64_t)k0 * m, c);
        KPCG_LAUNCHED("nys_proj_kernel");
    }
    sum_splits_kernel<<<(unsigned)((c * m + 255) / 256), 256, 0, st>>>(part, nsplit, c * m, w);
    KPCG_LAUNCHED("sum_splits_kernel");
    tri_lower_apply_kernel<<<dim3((unsigned)((m + 31) / 32), c), 1024, 0, st>>>(P.U.p, m, w, y);
    KPCG_LAUNCHED("tri_lower_apply_kernel");
    tri_upper_apply_kernel<<<dim3((unsigned)((m * 32 + 255) / 256), c), 256, 0, st>>>(P.U.p, m, y,
                                                                                     w);
    KPCG_LAUNCHED("tri_upper_apply_kernel");
    const size_t smem = sizeof(double) * (size_t)m * c;
    if (smem > 200 * 1024) fail(KPCG_ERR_ARG, "Nystrom apply: m * c too large");
    if (smem > 48 * 1024) raise_smem_limit((const void*)nys_back_kernel<T>, smem);
    int blocks = (int)std::min<int64_t>((n + 7) / 8, 152 * 16);
    nys_back_kernel<T><<<blocks, 256, smem, st>>>(P.KXU.p, n, m, w, c, R, ldr, Z, ldz,
                                                  1.0 / P.apply_noise);
    KPCG_LAUNCHED("nys_back_kernel");
}

// u = M^{-1} K_UX r for c columns (FP64 in and out, column-major, ld m for u).
void nystrom_project_solve(const PrecondState& P, const double* R, int64_t ldr, int c, double* u,
                           cudaStream_t st) {
    const int64_t n = P.n, m = P.m;
    const int64_t ablk = (m + 255) / 256;
    int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((152 * 4 + ablk - 1) / ablk,
                                                             (n + 127) / 128));
    const int64_t rps = (n + nsplit - 1) / nsplit;
    nsplit = (int)((n + rps - 1) / rps);
    double* part = const_cast<PrecondState&>(P).wpart.need((size_t)nsplit * c * m);
    double* w = const_cast<PrecondState&>(P).w.need((size_t)c * m);
    double* y = const_cast<PrecondState&>(P).y.need((size_t)c * m);
    for (int k0 = 0; k0 < c; k0 += PC) {
        const int nc = std::min(PC, c - k0);
        dim3 g((unsigned)((m + 255) / 256), (unsigned)nsplit);
        nys_proj_kernel<double><<<g, 256, 0, st>>>(P.KXU.p, n, m, R + (int64_t)k0 * ldr, ldr, nc,
                                                   rps, part + (int64_t)k0 * m, c);
        KPCG_LAUNCHED("nys_proj_kernel");
    }
    sum_splits_kernel<<<(unsigned)((c * m + 255) / 256), 256, 0, st>>>(part, nsplit, c * m, w);
    KPCG_LAUNCHED("sum_splits_kernel");
    tri_lower_apply_kernel<<<dim3((unsigned)((m + 31) / 32), c), 1024, 0, st>>>(P.U.p, m, w, y);
    KPCG_LAUNCHED("tri_lower_apply_kernel");
    tri_upper_apply_kernel<<<dim3((unsigned)((m * 32 + 255) / 256), c), 256, 0, st>>>(P.U.p, m, y,
                                                                                     u);
    KPCG_LAUNCHED("tri_upper_apply_kernel");
}

// out[i] = sum_a K_XU[i][a] u[a] (one column, FP64 accumulation, warp per row).
__global__ void nys_expand_kernel(const float2* __restrict__ KXU, int64_t n, int64_t m,
                                  const double* __restrict__ u, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const float2* Ki = KXU + i * m;
        double acc = 0.0;
        for (int64_t a = lane; a < m; a += 32) {
            const float2 kv = __ldg(Ki + a);
            acc = fma((double)kv.x + (double)kv.y, __ldg(u + a), acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) out[i] = acc;
    }
}

void nystrom_expand(const PrecondState& P, const double* u, double* out, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((P.n + 7) / 8, 152 * 16);
    nys_expand_kernel<<<blocks, 256, 0, st>>>(P.KXU.p, P.n, P.m, u, out);
    KPCG_LAUNCHED("nys_expand_kernel");
}

template <typename T>
static void bj_apply(const PrecondState& P, const T* R, int64_t ldr, int c, T* Z, int64_t ldz,
                     cudaStream_t st) {
    const int64_t nb = (P.n + P.b - 1) / P.b;
    const size_t smem = sizeof(double) * 2 * (size_t)P.b;
    if (smem > 48 * 1024) raise_smem_limit((const void*)bj_apply_kernel<T>, smem);
    bj_apply_kernel<T><<<dim3((unsigned)nb, c), 256, smem, st>>>(P.U.p, P.n, P.b, R, ldr, Z, ldz);
    KPCG_LAUNCHED("bj_apply_kernel");
}

template <typename T>
__global__ void scale_rows_kernel(T* __restrict__ dst, int64_t ldd, const T* __restrict__ src,
                                  int64_t lds, const double* __restrict__ sc, int64_t n) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i + (int64_t)k * ldd] = (T)((double)src[i + (int64_t)k * lds] * sc[i]);
}

template <typename T>
static T* fitc_tmp(const PrecondState& P, size_t count);
template <>
double* fitc_tmp<double>(const PrecondState& P, size_t count) {
    return const_cast<PrecondState&>(P).tmp64.need(count);
}
template <>
float* fitc_tmp<float>(const PrecondState& P, size_t count) {
    return const_cast<PrecondState&>(P).tmp32.need(count);
}

// FITC: z = D^{-1/2} Nys(D^{-1/2} r) with the unit-noise apply on the scaled K_XU.
template <typename T>
static void fitc_apply(const PrecondState& P, const T* R, int64_t ldr, int c, T* Z, int64_t ldz,
                       cudaStream_t st) {
    const int64_t n = P.n;
    T* tmp = fitc_tmp<T>(P, (size_t)n * c);
    const dim3 g((unsigned)std::min<int64_t>((n + 255) / 256, 1024), (unsigned)c);
    scale_rows_kernel<T><<<g, 256, 0, st>>>(tmp, n, R, ldr, P.dscale.p, n);
    KPCG_LAUNCHED("scale_rows_kernel");
    nystrom_apply<T>(P, tmp, n, c, Z, ldz, st);
    scale_rows_kernel<T><<<g, 256, 0, st>>>(Z, ldz, Z, ldz, P.dscale.p, n);
    KPCG_LAUNCHED("scale_rows_kernel");
}

namespace {

// One triangular factor of D^{-1} per block and column (one CTA each), U = L^{-T}
// per block: forward out_i = (L^{-1} in)_i = sum_{j <= i} U[j][i] in_j; backward
// out_j = (L^{-T} in)_j = sum_{i >= j} U[j][i] in_i.  The block is staged in
// shared memory first, so out may alias in.
template <typename T, bool FORWARD>
__global__ void pitc_tri_kernel(const double* __restrict__ Ub, int64_t n, int64_t b, const T* in,
                                int64_t ldi, T* out, int64_t ldo) {
    extern __shared__ double sv[];  // b
    const int64_t q = blockIdx.x;
    const int k = blockIdx.y;
    const int64_t bq = bsize(q, b, n);
    const int64_t r0 = q * b;
    const double* U = Ub + q * b * b;
    for (int64_t i = threadIdx.x; i < bq; i += blockDim.x)
        sv[i] = (double)in[r0 + i + (int64_t)k * ldi];
    __syncthreads();
    if (FORWARD) {
        for (int64_t i = threadIdx.x; i < bq; i += blockDim.x) {
            double s = 0.0;
            for (int64_t j = 0; j <= i; ++j) s = fma(U[j * bq + i], sv[j], s);
            out[r0 + i + (int64_t)k * ldo] = (T)s;
        }
    } else {
        const int lane = threadIdx.x & 31;
        const int nw = blockDim.x >> 5;
        for (int64_t j = threadIdx.x >> 5; j < bq; j += nw) {
            const double* Uj = U + j * bq;
            double s = 0.0;
            for (int64_t i = j + lane; i < bq; i += 32) s = fma(Uj[i], sv[i], s);
            s = warp_sum(s);
            if (lane == 0) out[r0 + j + (int64_t)k * ldo] = (T)s;
        }
    }
}

}  // namespace

// PITC: z = L_D^{-T} Nys(L_D^{-1} r) with the unit-noise apply on K~ = L_D^{-1} K_XU
// (D^{-1} = L_D^{-T} L_D^{-1}; the inversion lemma with D in place of noise I).
template <typename T>
static void pitc_apply(const PrecondState& P, const T* R, int64_t ldr, int c, T* Z, int64_t ldz,
                       cudaStream_t st) {
    const int64_t n = P.n, b = P.b;
    const int64_t nb = (n + b - 1) / b;
    T* tmp = fitc_tmp<T>(P, (size_t)n * c);
    const size_t smem = sizeof(double) * (size_t)b;
    if (smem > 48 * 1024) fail(KPCG_ERR_ARG, "PITC block too large");
    pitc_tri_kernel<T, true><<<dim3((unsigned)nb, (unsigned)c), 256, smem, st>>>(P.dinv.p, n, b,
                                                                               R, ldr, tmp, n);
    KPCG_LAUNCHED("pitc_tri_kernel");
    nystrom_apply<T>(P, tmp, n, c, Z, ldz, st);
    pitc_tri_kernel<T, false><<<dim3((unsigned)nb, (unsigned)c), 256, smem, st>>>(P.dinv.p, n, b,
                                                                                Z, ldz, Z, ldz);
    KPCG_LAUNCHED("pitc_tri_kernel");
}

template <typename T>
static void apply_any(const PrecondState& P, const T* R, int64_t ldr, int c, T* Z, int64_t ldz,
                      cudaStream_t st) {
    if ((P.kind == KPCG_PREC_NYSTROM || P.kind == KPCG_PREC_SPECTRAL) && P.ready)
        nystrom_apply<T>(P, R, ldr, c, Z, ldz, st);
    else if (P.kind == KPCG_PREC_FITC && P.ready)
        fitc_apply<T>(P, R, ldr, c, Z, ldz, st);
    else if (P.kind == KPCG_PREC_PITC && P.ready)
        pitc_apply<T>(P, R, ldr, c, Z, ldz, st);
    else if (P.kind == KPCG_PREC_BLOCK_JACOBI && P.ready)
        bj_apply<T>(P, R, ldr, c, Z, ldz, st);
    else
        copy_cols<T>(Z, ldz, R, ldr, P.n, c, st);
}

void precond_apply_f64(const PrecondState& P, const double* R, int64_t ldr, int c, double* Z,
                       int64_t ldz, cudaStream_t st) {
    apply_any<double>(P, R, ldr, c, Z, ldz, st);
}
void precond_apply_f32(const PrecondState& P, const float* R, int64_t ldr, int c, float* Z,
                       int64_t ldz, cudaStream_t st) {
    apply_any<float>(P, R, ldr, c, Z, ldz, st);
}


// ------------------------------------------------------------------------
// Batched Nystrom apply over many problems (batch layout: problem p owns
// columns p*c .. p*c+c-1).  Same arithmetic as the single-problem apply:
// w = K_UX r with Dot2 on FP32 pairs, y = L^{-1} w, u = L^{-T} y (FP64),
// z = (r - K_XU u) / sigma^2 with FP64 accumulation.  Grids carry the problem
// index; blocks past a problem's sizes, and problems with no active column,
// return at once.
namespace {

constexpr int kSplitRows = 512;
constexpr int kRb = 8;  // rows (projection) or row chunks (back product) loaded per batch

__device__ __forceinline__ bool nb_live(const int* __restrict__ active, int p, int c) {
    if (!active) return true;
    for (int k = 0; k < c; ++k)
        if (active[p * c + k]) return true;
    return false;
}

// part[pbase + (split * c + k) * m + a] for columns k0 .. k0+ncols-1 (ncols <= NC)
template <int NC>
__global__ void __launch_bounds__(256)
    nys_batch_proj_kernel(const NysBatchProb* __restrict__ probs, int c, const float* __restrict__ R,
                          int64_t ldr, int k0, int ncols, const int* __restrict__ active,
                          double* __restrict__ part) {
    __shared__ float sr[128][NC];
    const int p = blockIdx.z;
    const NysBatchProb pb = probs[p];
    if (pb.m == 0 || (int)blockIdx.y >= pb.nsplit || (int64_t)blockIdx.x * 256 >= pb.m ||
        !nb_live(active, p, c))
        return;
    const int64_t m = pb.m;
    const int64_t a = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * pb.rows_per_split;
    const int64_t r1 = min(pb.n, r0 + pb.rows_per_split);
    const float* Rp = R + ((int64_t)p * c + k0) * ldr;
    Acc2 acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = {0.f, 0.f};
    for (int64_t rs = r0; rs < r1; rs += 128) {
        __syncthreads();
        for (int e = threadIdx.x; e < 128 * NC; e += 256) {
            const int k = e / 128, r = e % 128;
            sr[r][k] = (rs + r < r1 && k < ncols) ? Rp[rs + r + (int64_t)k * ldr] : 0.f;
        }
        __syncthreads();
        const int rn = (int)min((int64_t)128, r1 - rs);
        if (a < m) {
            const float2* Kp = pb.KXU + rs * m + a;
            // batches of kRb rows: their loads are issued before any is used, so
            // each thread keeps kRb * 8 bytes of K_XU in flight (the pass is
            // bound by HBM latency times the bytes in flight, not by the Dot2)
            int r = 0;
            for (; r + kRb <= rn; r += kRb) {
                float2 kv[kRb];
#pragma unroll
                for (int u = 0; u < kRb; ++u) kv[u] = __ldg(Kp + (int64_t)(r + u) * m);
#pragma unroll
                for (int u = 0; u < kRb; ++u)
#pragma unroll
                    for (int k = 0; k < NC; ++k)
                        if (k < ncols) {
                            dot2_add(acc[k], kv[u].x, sr[r + u][k]);
                            acc[k].c = fmaf(kv[u].y, sr[r + u][k], acc[k].c);
                        }
            }
            for (; r < rn; ++r) {
                const float2 kv = __ldg(Kp + (int64_t)r * m);
#pragma unroll
                for (int k = 0; k < NC; ++k)
                    if (k < ncols) {
                        dot2_add(acc[k], kv.x, sr[r][k]);
                        acc[k].c = fmaf(kv.y, sr[r][k], acc[k].c);
                    }
            }
        }
    }
    if (a < m) {
#pragma unroll
        for (int k = 0; k < NC; ++k)
            if (k < ncols)
                part[pb.pbase + ((int64_t)blockIdx.y * c + k0 + k) * m + a] =
                    (double)acc[k].s + (double)acc[k].c;
    }
}

// w = sum of the split partials: a warp per entry (lanes stride over the
// splits, then a fixed-order warp sum), so the dependent FP64 adds of one
// entry are ~nsplit / 32 instead of nsplit.
__global__ void nys_batch_sum_kernel(const NysBatchProb* __restrict__ probs, int c,
                                     const int* __restrict__ active,
                                     const double* __restrict__ part, double* __restrict__ w) {
    const int p = blockIdx.y;
    const NysBatchProb pb = probs[p];
    const int64_t len = (int64_t)c * pb.m;
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= len || !nb_live(active, p, c)) return;
    double s = 0.0;
    for (int sp = lane; sp < pb.nsplit; sp += 32) s += part[pb.pbase + (int64_t)sp * len + e];
    s = warp_sum(s);
    if (lane == 0) w[pb.wbase + e] = s;
}

// y = L^{-1} w per problem and column (same scheme as tri_lower_apply_kernel).
// A bounded grid walks the flat list of (problem, column, 32-row block)
// items, so items of finished problems cost a flag test, not a CTA.
__global__ void __launch_bounds__(1024)
    nys_batch_lower_kernel(const NysBatchProb* __restrict__ probs, int c,
                           const int* __restrict__ active, const int4* __restrict__ items,
                           int nitems, const double* __restrict__ w, double* __restrict__ y) {
    __shared__ double part[32][33];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 wk = items[it];
        const int p = wk.x, k = wk.y;
        if (!nb_live(active, p, c)) continue;  // uniform over the block
        const NysBatchProb& pb = probs[p];
        const int64_t m = pb.m;
        const int64_t i = (int64_t)wk.z * 32 + lane;
        const double* wk_ = w + pb.wbase + (int64_t)k * m;
        double s = 0.0;
        if (i < m)
            for (int64_t j = g; j <= i; j += 32) s = fma(pb.U[j * m + i], wk_[j], s);
        part[g][lane] = s;
        __syncthreads();
        if (g == 0 && i < m) {
            double t = 0.0;
            for (int q = 0; q < 32; ++q) t += part[q][lane];
            y[pb.wbase + (int64_t)k * m + i] = t;
        }
        __syncthreads();
    }
}

// u = L^{-T} y (warp per entry; items of 8 entries), written over w and as
// FP32 pairs (hi, lo)
__global__ void nys_batch_upper_kernel(const NysBatchProb* __restrict__ probs, int c,
                                       const int* __restrict__ active,
                                       const int4* __restrict__ items, int nitems,
                                       const double* __restrict__ y, double* __restrict__ u,
                                       float2* __restrict__ u2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 wk = items[it];
        const int p = wk.x, k = wk.y;
        const NysBatchProb& pb = probs[p];
        const int64_t m = pb.m;
        const int64_t j = (int64_t)wk.z * 8 + warp;
        if (j >= m || !nb_live(active, p, c)) continue;
        const double* yk = y + pb.wbase + (int64_t)k * m;
        const double* Uj = pb.U + j * m;
        double s = 0.0;
        for (int64_t i = j + lane; i < m; i += 32) s = fma(Uj[i], yk[i], s);
        s = warp_sum(s);
        if (lane == 0) {
            u[pb.wbase + (int64_t)k * m + j] = s;
            const float hi = (float)s;
            u2[pb.wbase + (int64_t)k * m + j] = make_float2(hi, (float)(s - (double)hi));
        }
    }
}

// z = (r - K_XU u) / sigma^2 (warp per row, all columns k0 .. k0+ncols-1 of
// the problem in one sweep over the row of K_XU), zero past n_p; m = 0 means
// no preconditioner (z = r).  Problems with no active column are left as they
// are: the CG does not read those columns again.
//
// u can hold entries ~1e6 that cancel to O(1) in K_XU u (the Nystrom P^{-1}
// spans ~1/sigma^2 .. 1/lambda_max), so the sum needs ~FP64 accuracy; FP64
// itself runs at 1/64 of the FP32 rate here.  Both factors are FP32 pairs
// (hi, lo); each term is split exactly (TwoProduct by FMA, plus the two
// cross terms) and summed with TwoSum (Dot2, Ogita-Rump-Oishi 2005), about
// 2^-46 relative per term at ~11 FP32 operations.
// With STAGE the problem's u (ncols x m pairs) is first copied to shared
// memory: every row of the block reads all of it.
template <int NC, bool STAGE>
__global__ void __launch_bounds__(256)
    nys_batch_back_kernel(const NysBatchProb* __restrict__ probs, int c, int k0, int ncols,
                          const int* __restrict__ active, const float2* __restrict__ u,
                          const float* __restrict__ R, int64_t ldr, float* __restrict__ Z,
                          int64_t ldz, int64_t nrows) {
    extern __shared__ float2 su2[];
    const int p = blockIdx.y;
    const NysBatchProb pb = probs[p];
    if (!nb_live(active, p, c)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float* Rp = R + ((int64_t)p * c + k0) * ldr;
    float* Zp = Z + ((int64_t)p * c + k0) * ldz;
    const float2* up = u + pb.wbase + (int64_t)k0 * pb.m;
    if constexpr (STAGE) {
        for (int64_t e = threadIdx.x; e < (int64_t)ncols * pb.m; e += blockDim.x) su2[e] = up[e];
        __syncthreads();
        up = su2;
    }
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nrows;
         i += warps) {
        if (i >= pb.n || pb.m == 0) {
            for (int k = lane; k < ncols; k += 32)
                Zp[i + (int64_t)k * ldz] = (i < pb.n) ? Rp[i + (int64_t)k * ldr] : 0.f;
            continue;
        }
        const float2* Ki = pb.KXU + i * pb.m;
        Acc2 acc[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] = {0.f, 0.f};
        // the row in batches of kRb chunks of 32 entries, all loads of a batch
        // issued before any is used (bytes in flight, as in the projection)
        for (int64_t a0 = lane; a0 < pb.m; a0 += 32 * kRb) {
            float2 kv[kRb];
#pragma unroll
            for (int u = 0; u < kRb; ++u) {
                const int64_t a = a0 + 32 * u;
                kv[u] = (a < pb.m) ? __ldg(Ki + a) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kRb; ++u) {
                const int64_t a = a0 + 32 * u;
                if (a >= pb.m) break;
#pragma unroll
                for (int k = 0; k < NC; ++k)
                    if (k < ncols) {
                        const float2 uv = up[(int64_t)k * pb.m + a];
                        dot2_add(acc[k], kv[u].x, uv.x);
                        acc[k].c = fmaf(kv[u].x, uv.y, fmaf(kv[u].y, uv.x, acc[k].c));
                    }
            }
        }
        // warp sum of the pairs with TwoSum on every step (FP64 adds would
        // hold the FP64 pipe, ~1/64 rate, longer than the whole sweep above)
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (k < ncols) {
                float hs = acc[k].s, hc = acc[k].c;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float os = __shfl_xor_sync(0xffffffffu, hs, o);
                    const float oc = __shfl_xor_sync(0xffffffffu, hc, o);
                    const float t = hs + os;
                    const float z = t - hs;
                    const float e = (hs - (t - z)) + (os - z);
                    hs = t;
                    hc = hc + oc + e;
                }
                if (lane == 0) {
                    // z = (r - (hs + hc)) / sigma^2: r - hs by TwoSum, then the tails
                    const float r = Rp[i + (int64_t)k * ldr];
                    const float d = r - hs;
                    const float bv = d - r;
                    const float de = (r - (d - bv)) + (-hs - bv);
                    Zp[i + (int64_t)k * ldz] = (d + (de - hc)) * pb.inv_noise_f;
                }
            }
        }
    }
}

}  // namespace


void nys_batch_plan(NysBatch& nb, const std::vector<const PrecondState*>& Ps, int c,
                    cudaStream_t st) {
    nb.P = (int)Ps.size();
    nb.c = c;
    nb.hprobs.assign((size_t)nb.P, NysBatchProb{});
    nb.mmax = 0;
    nb.wtotal = 0;
    nb.ptotal = 0;
    nb.nsplit_max = 1;
    for (int p = 0; p < nb.P; ++p) {
        const PrecondState& P = *Ps[(size_t)p];
        NysBatchProb& q = nb.hprobs[(size_t)p];
        q.n = P.n;
        const bool on =
            P.ready && (P.kind == KPCG_PREC_NYSTROM || P.kind == KPCG_PREC_SPECTRAL);
        q.m = on ? P.m : 0;
        q.KXU = on ? P.KXU.p : nullptr;
        q.U = on ? P.U.p : nullptr;
        q.inv_noise = on ? 1.0 / P.apply_noise : 1.0;
        q.inv_noise_f = (float)q.inv_noise;
        q.rows_per_split = kSplitRows;
        q.nsplit = (int32_t)std::max<int64_t>(1, (P.n + kSplitRows - 1) / kSplitRows);
        q.wbase = nb.wtotal;
        q.pbase = nb.ptotal;
        nb.wtotal += (int64_t)c * q.m;
        nb.ptotal += (int64_t)q.nsplit * c * q.m;
        nb.mmax = std::max(nb.mmax, q.m);
        nb.nsplit_max = std::max(nb.nsplit_max, (int)q.nsplit);
    }
    std::vector<int4> L, U;
    for (int p = 0; p < nb.P; ++p) {
        const int64_t m = nb.hprobs[(size_t)p].m;
        for (int k = 0; k < c; ++k) {
            for (int64_t ib = 0; ib * 32 < m; ++ib) L.push_back(make_int4(p, k, (int)ib, 0));
            for (int64_t jb = 0; jb * 8 < m; ++jb) U.push_back(make_int4(p, k, (int)jb, 0));
        }
    }
    nb.nL = (int)L.size();
    nb.nU = (int)U.size();
    nb.itemsL.need(std::max<size_t>(1, L.size()));
    nb.itemsU.need(std::max<size_t>(1, U.size()));
    if (!L.empty())
        KPCG_CUDA(cudaMemcpyAsync(nb.itemsL.p, L.data(), sizeof(int4) * L.size(),
                                  cudaMemcpyHostToDevice, st));
    if (!U.empty())
        KPCG_CUDA(cudaMemcpyAsync(nb.itemsU.p, U.data(), sizeof(int4) * U.size(),
                                  cudaMemcpyHostToDevice, st));
    nb.probs.need(nb.hprobs.size());
    nb.part.need((size_t)std::max<int64_t>(1, nb.ptotal));
    nb.w.need((size_t)std::max<int64_t>(1, nb.wtotal));
    nb.y.need((size_t)std::max<int64_t>(1, nb.wtotal));
    nb.u2.need((size_t)std::max<int64_t>(1, nb.wtotal));
    KPCG_CUDA(cudaMemcpyAsync(nb.probs.p, nb.hprobs.data(), sizeof(NysBatchProb) * nb.hprobs.size(),
                              cudaMemcpyHostToDevice, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
}

void nys_batch_apply(NysBatch& nb, const float* R, int64_t ldr, float* Z, int64_t ldz,
                     int64_t nrows, const int* active, cudaStream_t st) {
    if (nb.P == 0) return;
    const int c = nb.c;
    if (nb.mmax > 0) {
        const unsigned ablk = (unsigned)((nb.mmax + 255) / 256);
        const dim3 g(ablk, (unsigned)nb.nsplit_max, (unsigned)nb.P);
        for (int k0 = 0; k0 < c; k0 += 16) {
            const int nc = std::min(16, c - k0);
            if (nc <= 4)
                nys_batch_proj_kernel<4><<<g, 256, 0, st>>>(nb.probs.p, c, R, ldr, k0, nc, active,
                                                           nb.part.p);
            else if (nc <= 8)
                nys_batch_proj_kernel<8><<<g, 256, 0, st>>>(nb.probs.p, c, R, ldr, k0, nc, active,
                                                           nb.part.p);
            else if (nc <= 9)
                nys_batch_proj_kernel<9><<<g, 256, 0, st>>>(nb.probs.p, c, R, ldr, k0, nc, active,
                                                           nb.part.p);
            else
                nys_batch_proj_kernel<16><<<g, 256, 0, st>>>(nb.probs.p, c, R, ldr, k0, nc, active,
                                                            nb.part.p);
            KPCG_LAUNCHED("nys_batch_proj_kernel");
        }
        nys_batch_sum_kernel<<<dim3((unsigned)((c * nb.mmax + 7) / 8), (unsigned)nb.P), 256, 0,
                               st>>>(nb.probs.p, c, active, nb.part.p, nb.w.p);
        KPCG_LAUNCHED("nys_batch_sum_kernel");
        nys_batch_lower_kernel<<<(unsigned)std::max(1, std::min(nb.nL, 2 * 152)), 1024, 0,
                                 st>>>(nb.probs.p, c, active, nb.itemsL.p, nb.nL, nb.w.p,
                                       nb.y.p);
        KPCG_LAUNCHED("nys_batch_lower_kernel");
        nys_batch_upper_kernel<<<(unsigned)std::max(1, std::min(nb.nU, 8 * 152)), 256, 0,
                                 st>>>(nb.probs.p, c, active, nb.itemsU.p, nb.nU, nb.y.p, nb.w.p,
                                       nb.u2.p);
        KPCG_LAUNCHED("nys_batch_upper_kernel");
    }
    // rows per problem: at least ~16 warps per SM over the whole batch
    const unsigned blocks =
        (unsigned)std::min<int64_t>((nrows + 7) / 8, std::max(256, 152 * 16 / std::max(1, nb.P)));
    for (int k0 = 0; k0 < c; k0 += 16) {
        const int nc = std::min(16, c - k0);
        const dim3 g(blocks, (unsigned)nb.P);
        const size_t smem = sizeof(float2) * (size_t)nc * (size_t)nb.mmax;
        const bool stage = smem <= 200 * 1024;
        auto go = [&](auto kern) {
            if (stage && smem > 48 * 1024) raise_smem_limit((const void*)kern, smem);
            kern<<<g, 256, stage ? smem : 0, st>>>(nb.probs.p, c, k0, nc, active, nb.u2.p, R, ldr,
                                                   Z, ldz, nrows);
        };
        if (nc <= 4)
            stage ? go(nys_batch_back_kernel<4, true>) : go(nys_batch_back_kernel<4, false>);
        else if (nc <= 8)
            stage ? go(nys_batch_back_kernel<8, true>) : go(nys_batch_back_kernel<8, false>);
        else if (nc <= 9)
            stage ? go(nys_batch_back_kernel<9, true>) : go(nys_batch_back_kernel<9, false>);
        else
            stage ? go(nys_batch_back_kernel<16, true>) : go(nys_batch_back_kernel<16, false>);
        KPCG_LAUNCHED("nys_batch_back_kernel");
    }
}

}  // namespace kpcg
