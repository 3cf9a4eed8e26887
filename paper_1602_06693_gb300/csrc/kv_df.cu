// Double-float K.V: FP64-class kernel products on the FP32 pipe.
//
// GB300 issues FP32 at 64 times its FP64 rate, and an FP64 K.V at n = 65536
// is bound by that FP64 rate.  This kernel carries every quantity of an entry
// K_ij = s^2 exp(-1/2 sum_r (x_ir - x_jr)^2 / l_r^2) (Eq. 1) as an unevaluated
// sum of two FP32 numbers (hi + lo), which keeps about 44 bits:
//
//  * Inputs.  x' = (x - mu) / l * sqrt(log2(e)/2) (FP64) is split per
//    dimension r into hi, a multiple of 2^(k_r - 23) with |x'| < 2^k_r (so
//    hi_i - hi_j is exact in FP32), lo = fl(x' - hi) and lo2 = fl(x' - hi - lo):
//    the three parts hold the FP64 value exactly, so the only per-point error
//    is the FP64 rounding of x' itself.  (With two parts, the 2^-48 rounding of
//    lo is a per-point, hence structured, perturbation of K; multiplied by a
//    solution with |alpha| >> |y| it limited the residual to about 1e-7.)
//  * Squared distance.  delta = D + E with D = hi_i - hi_j exact, E = (lo_i -
//    lo_j) + (lo2_i - lo2_j); delta^2 = D*D (split exactly by an FMA,
//    "TwoProduct") + 2 D E + E^2,
//    accumulated into the exponent a = log2(s^2) - |x'_i - x'_j|^2 with Knuth's
//    TwoSum, so no rounding of the running sum is lost.
//  * exp2 of a double-float (table-driven method of P. T. P. Tang, "Table-
//    driven implementation of the exponential function", 1989): a = k + j/256
//    + r, 2^a = 2^k * 2^(j/256) * e^(r ln 2); the 257 values 2^(j/256) are a
//    double-float table computed on the host in FP64, e^t for |t| < 0.0014 is
//    1 + t + t^2 (1/2 + t (1/6 + t/24)) with the linear part in double-float.
//  * Contraction.  V (FP64) enters as hi + lo; products are split exactly and
//    summed with TwoSum (Ogita-Rump-Oishi style), partial sums leave as FP64.
//
// Rows: one per thread; column tiles of the operands staged in shared memory;
// column ranges split across CTAs and added in FP64 by a second kernel in a
// fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "df_arith.cuh"

namespace kpcg {
namespace {

constexpr int KT = 256;
constexpr int TJ = 64;

int sm_count_df() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        if (cached <= 0) cached = 148;
    }
    return cached;
}

template <int DP, int CB>
__global__ void __launch_bounds__(KT)
    kv_df_kernel(const float4* __restrict__ xs, int64_t n, float c0h, float c0l,
                 const double* __restrict__ V, int64_t ldv, int ncols,
                 const float2* __restrict__ gtab, double* __restrict__ part, int64_t ldp,
                 int64_t cps) {
    __shared__ float2 tab[NTAB];
    __shared__ float4 sx[TJ * DP];
    __shared__ float2 sv[TJ * CB];
    for (int e = threadIdx.x; e < NTAB; e += KT) tab[e] = gtab[e];
    const int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * cps;
    const int64_t j1 = min(n, j0 + cps);
    float4 xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < n) ? xs[i * DP + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    float S[CB], C[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) S[k] = C[k] = 0.f;
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        const int jn = (int)min((int64_t)TJ, j1 - jt);
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DP; e += KT) {
            const int jj = e / DP;
            sx[e] = (jj < jn) ? xs[(jt + jj) * DP + (e - jj * DP)] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = threadIdx.x; e < TJ * CB; e += KT) {
            const int k = e / TJ, jj = e - k * TJ;
            double v = (jj < jn && k < ncols) ? V[(jt + jj) + (int64_t)k * ldv] : 0.0;
            const float vh = (float)v;
            sv[jj * CB + k] = make_float2(vh, (float)(v - (double)vh));
        }
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            float ah = c0h, al = c0l;
#pragma unroll
            for (int q = 0; q < DP; ++q) {
                const float4 xj = sx[jj * DP + q];
                const float D = xi[q].x - xj.x;  // exact
                const float E = (xi[q].y - xj.y) + (xi[q].z - xj.z);
                const float P = D * D;
                float Pe = fmaf(D, D, -P);
                Pe = fmaf(2.f * D, E, Pe);
                Pe = fmaf(E, E, Pe);
                df_sub(ah, al, P, Pe);
            }
            const DF e = df_exp2(ah, al, tab);
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const float2 v = sv[jj * CB + k];
                const float P = e.h * v.x;
                float Pe = fmaf(e.h, v.x, -P);
                Pe = fmaf(e.h, v.y, Pe);
                Pe = fmaf(e.l, v.x, Pe);
                df_acc(S[k], C[k], P, Pe);
            }
            if ((jj & 31) == 31)
#pragma unroll
                for (int k = 0; k < CB; ++k) df_renorm(S[k], C[k]);
        }
    }
    if (i < n) {
#pragma unroll
        for (int k = 0; k < CB; ++k)
            if (k < ncols) part[((int64_t)blockIdx.y * CB + k) * ldp + i] = (double)S[k] + (double)C[k];
    }
}


// ---------------------------------------------------------------------------
// Symmetric variant: K is symmetric, so each entry of an off-diagonal 128 x 128
// tile pair (I, J), I < J, is evaluated once and used twice: for the row sums
// of tile I (thread-owned rows, as above) and, through a shared-memory
// transpose of the products e_ij v_i, for the column sums of tile J.  A CTA
// walks a run of J tiles for one I.  Row partials go to prow[I][chunk], column
// partials to pcol[J][I]; a second kernel adds them in a fixed order.
constexpr int ST = 128;   // tile edge
constexpr int SCW = 32;   // columns per transpose chunk

template <int DP, int CB>
__global__ void __launch_bounds__(ST)
    kv_df_sym_kernel(const float4* __restrict__ xs, int64_t n, int nt, float c0h, float c0l,
                     const double* __restrict__ V, int64_t ldv, int ncols,
                     const float2* __restrict__ gtab, const int4* __restrict__ work, int G,
                     int nchunk, double* __restrict__ prow, double* __restrict__ pcol) {
    // dynamic shared memory: x_J tile, exp2 table, V_J, transpose buffer, reductions
    extern __shared__ float4 dsm[];
    float4* sx = dsm;                                                    // ST * DP
    float2* tab = reinterpret_cast<float2*>(sx + ST * DP);               // NTAB (+1 pad)
    float2* sv = tab + NTAB + 1;                                         // ST * CB
    float2 (*W)[ST][SCW + 1] = reinterpret_cast<float2 (*)[ST][SCW + 1]>(sv + ST * CB);
    float2 (*red)[4][SCW] = reinterpret_cast<float2 (*)[4][SCW]>(&W[CB][0][0]);
    for (int e = threadIdx.x; e < NTAB; e += ST) tab[e] = gtab[e];
    const int4 wk = work[blockIdx.x];  // (I, J0, J1, chunk)
    const int I = wk.x;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int64_t i = (int64_t)I * ST + t;
    float4 xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q)
        xi[q] = (i < n) ? xs[i * DP + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    float2 vi[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        const double v = (i < n && k < ncols) ? V[i + (int64_t)k * ldv] : 0.0;
        const float vh = (float)v;
        vi[k] = make_float2(vh, (float)(v - (double)vh));
    }
    float S[CB], C[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) S[k] = C[k] = 0.f;
    for (int J = wk.y; J < wk.z; ++J) {
        __syncthreads();
        for (int e = t; e < ST * DP; e += ST) {
            const int jj = e / DP;
            const int64_t j = (int64_t)J * ST + jj;
            sx[e] = (j < n) ? xs[j * DP + (e - jj * DP)] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = t; e < ST * CB; e += ST) {
            const int k = e / ST, jj = e - k * ST;
            const int64_t j = (int64_t)J * ST + jj;
            const double v = (j < n && k < ncols) ? V[j + (int64_t)k * ldv] : 0.0;
            const float vh = (float)v;
            sv[jj * CB + k] = make_float2(vh, (float)(v - (double)vh));
        }
        __syncthreads();
        const bool mirror = (J != I);
        for (int c0 = 0; c0 < ST; c0 += SCW) {
            for (int jj = 0; jj < SCW; ++jj) {
                const int jc = c0 + jj;
                float ah = c0h, al = c0l;
#pragma unroll
                for (int q = 0; q < DP; ++q) {
                    const float4 xj = sx[jc * DP + q];
                    const float D = xi[q].x - xj.x;  // exact
                    const float E = (xi[q].y - xj.y) + (xi[q].z - xj.z);
                    const float P = D * D;
                    float Pe = fmaf(D, D, -P);
                    Pe = fmaf(D, E + E, Pe);
                    Pe = fmaf(E, E, Pe);
                    df_sub(ah, al, P, Pe);
                }
                const DF e = df_exp2(ah, al, tab);
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const float2 v = sv[jc * CB + k];
                    const float P = e.h * v.x;
                    float Pe = fmaf(e.h, v.x, -P);
                    Pe = fmaf(e.h, v.y, Pe);
                    Pe = fmaf(e.l, v.x, Pe);
                    df_acc(S[k], C[k], P, Pe);
                    if (mirror) {
                        const float Q = e.h * vi[k].x;
                        float Qe = fmaf(e.h, vi[k].x, -Q);
                        Qe = fmaf(e.h, vi[k].y, Qe);
                        Qe = fmaf(e.l, vi[k].x, Qe);
                        W[k][t][jj] = make_float2(Q, Qe);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) df_renorm(S[k], C[k]);
            if (mirror) {
                __syncthreads();
                // column sums: warp w adds rows 32w..32w+31 of column `lane`
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    float cs = 0.f, cc = 0.f;
                    for (int r = 0; r < 32; ++r) {
                        const float2 w = W[k][warp * 32 + r][lane];
                        df_acc(cs, cc, w.x, w.y);
                    }
                    red[k][warp][lane] = make_float2(cs, cc);
                }
                __syncthreads();
                if (warp == 0) {
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        float cs = 0.f, cc = 0.f;
#pragma unroll
                        for (int w = 0; w < 4; ++w) df_acc(cs, cc, red[k][w][lane].x, red[k][w][lane].y);
                        pcol[(((size_t)J * nt + I) * CB + k) * ST + c0 + lane] =
                            (double)cs + (double)cc;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CB; ++k)
        prow[(((size_t)I * nchunk + wk.w) * CB + k) * ST + t] = (double)S[k] + (double)C[k];
}


constexpr int NTAB64 = 256;  // 2^(j/256), j = 0..255, FP64

// e^a in FP64 by the table-driven method of P. T. P. Tang ("Table-driven
// implementation of the exponential function", 1989): a = m ln2/256 + r with
// m = rint(256 a / ln 2), read off the low word of 256 a / ln2 + 1.5 * 2^52;
// r = a - m ln2/256 with ln2/256 split so that the first product is exact,
// |r| <= ln2/512; e^a = 2^(m >> 8) * 2^((m & 255)/256) * e^r with e^r - 1 as
// its Taylor polynomial to r^5 (the next term is below 2^-66 relative), and
// the power of two added to the exponent field.  Arguments below -708 are
// clamped there (e^-708 ~ 3e-308 instead of a smaller number).  About 1 ulp;
// ten FP64 operations and one table read.
__device__ __forceinline__ double exp_tab64(double a, const double* __restrict__ tab) {
    a = fmax(a, -708.0);
    const double t = fma(a, 0x1.71547652b82fep+8, 6755399441055744.0);
    const int mi = __double2loint(t);
    const double mf = t - 6755399441055744.0;
    double r = fma(-mf, 0x1.62e42ff000000p-9, a);  // exact
    r = fma(-mf, -0x1.718432a1b0e26p-43, r);
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(r, q, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    q = fma(r, q, 1.0);
    const double T = tab[mi & (NTAB64 - 1)];
    const double e = fma(T, r * q, T);
    return __hiloint2double(__double2hiint(e) + ((mi >> 8) << 20), __double2loint(e));
}

// Native-FP64 symmetric variant (used for the FP64 residuals): the same tile
// pairs, transpose and reduction, entries exp(c0 - |x'_i - x'_j|^2) in FP64
// (the exp by exp_tab64).
template <int DP, int CB>
__global__ void __launch_bounds__(ST)
    kv_f64_sym_kernel(const double* __restrict__ xs, int64_t n, int nt, double c0,
                      const double* __restrict__ V, int64_t ldv, int ncols,
                      const int4* __restrict__ work, int G, int nchunk,
                      double* __restrict__ prow, double* __restrict__ pcol,
                      const double* __restrict__ gtab64) {
    extern __shared__ double dsm64[];
    double* sx = dsm64;                 // ST * DP
    double* sv = sx + ST * DP;          // ST * CB
    double (*W)[ST][SCW + 1] = reinterpret_cast<double (*)[ST][SCW + 1]>(sv + ST * CB);
    double (*red)[4][SCW] = reinterpret_cast<double (*)[4][SCW]>(&W[CB][0][0]);
    double* tab = &red[CB][0][0];       // NTAB64
    for (int e = threadIdx.x; e < NTAB64; e += blockDim.x) tab[e] = gtab64[e];
    const int4 wk = work[blockIdx.x];
    const int I = wk.x;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int64_t i = (int64_t)I * ST + t;
    double xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < n) ? xs[i * DP + q] : 0.0;
    double vi[CB], S[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        vi[k] = (i < n && k < ncols) ? V[i + (int64_t)k * ldv] : 0.0;
        S[k] = 0.0;
    }
    for (int J = wk.y; J < wk.z; ++J) {
        __syncthreads();
        for (int e = t; e < ST * DP; e += ST) {
            const int jj = e / DP;
            const int64_t j = (int64_t)J * ST + jj;
            sx[e] = (j < n) ? xs[j * DP + (e - jj * DP)] : 0.0;
        }
        for (int e = t; e < ST * CB; e += ST) {
            const int k = e / ST, jj = e - k * ST;
            const int64_t j = (int64_t)J * ST + jj;
            sv[jj * CB + k] = (j < n && k < ncols) ? V[j + (int64_t)k * ldv] : 0.0;
        }
        __syncthreads();
        const bool mirror = (J != I);
        for (int cst = 0; cst < ST; cst += SCW) {
            for (int jj = 0; jj < SCW; ++jj) {
                const int jc = cst + jj;
                double a = c0;
#pragma unroll
                for (int q = 0; q < DP; ++q) {
                    const double dlt = xi[q] - sx[jc * DP + q];
                    a = fma(-dlt, dlt, a);
                }
                const double e = exp_tab64(a, tab);
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    S[k] = fma(e, sv[jc * CB + k], S[k]);
                    if (mirror) W[k][t][jj] = e * vi[k];
                }
            }
            if (mirror) {
                __syncthreads();
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    double cs = 0.0;
                    for (int r = 0; r < 32; ++r) cs += W[k][warp * 32 + r][lane];
                    red[k][warp][lane] = cs;
                }
                __syncthreads();
                if (warp == 0) {
#pragma unroll
                    for (int k = 0; k < CB; ++k)
                        pcol[(((size_t)J * nt + I) * CB + k) * ST + cst + lane] =
                            ((red[k][0][lane] + red[k][1][lane]) + red[k][2][lane]) +
                            red[k][3][lane];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CB; ++k) prow[(((size_t)I * nchunk + wk.w) * CB + k) * ST + t] = S[k];
}


// ---------------------------------------------------------------------------
// Exact-difference FP32 product (the inner operator of KPCG_FP32X_IR).
//
// Rounding the scaled inputs x' to FP32 perturbs every point by ~2^-24: a
// perturbation that moves whole rows and columns of K together, so it acts on
// smooth vectors with the size of K's largest eigenvalue, and K_y^{-1} then
// multiplies it by up to 1/sigma^2 -- at n = 65536 and sigma^2 = 1e-4 the
// product of the two is ~8, and an FP32 inner solve cannot precondition the
// system.  Rounding errors that are independent per entry act like a random
// matrix instead, of norm ~ eps rms(K) sqrt(n), far below sigma^2.
// So this kernel keeps every per-point quantity exact and lets only the
// per-entry arithmetic round:
//  * x' arrives as the double-float pair (hi, lo) of kv_df_kernel (hi on a
//    per-dimension grid, so hi_i - hi_j is exact; lo carries the next 24 bits);
//    the difference is D + E rounded once, the squared distance sums in FP32;
//  * exp2 of the exponent: MUFU ex2.approx (EXPP = 0) or a degree-7 Taylor
//    polynomial of 2^f = e^(f ln 2), |f| <= 1/2, on the FMA pipe (EXPP = 1,
//    about one FP32 ulp);
//  * row sums with V are compensated (TwoSum into an FP32 pair), so the
//    accumulation adds no per-row error; the mirrored column sums of an
//    off-diagonal tile pair go through the shared-memory transpose of the
//    symmetric double-float kernel and are compensated the same way.
// V and O are FP32 (the inner PCG's vectors); partial sums leave as FP64.
template <int EXPP>
__device__ __forceinline__ float xf_exp2(float a) {
    if (EXPP == 0) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
        return y;
    } else {
        a = fmaxf(a, -125.f);
        const float big = a + 12582912.f;                  // 1.5 * 2^23: round to integer
        const int ki = __float_as_int(big) - 0x4B400000;
        const float f = a - (big - 12582912.f);           // exact, |f| <= 1/2
        // (ln 2)^k / k!, k = 7 .. 1
        float p = fmaf(f, 1.5252733804059840e-05f, 1.5403530393381608e-04f);
        p = fmaf(p, f, 1.3333558146428443e-03f);
        p = fmaf(p, f, 9.6181291076284772e-03f);
        p = fmaf(p, f, 5.5504108664821580e-02f);
        p = fmaf(p, f, 2.4022650695910071e-01f);
        p = fmaf(p, f, 6.9314718055994531e-01f);
        p = fmaf(p, f, 1.f);
        return __int_as_float(__float_as_int(p) + (ki << 23));
    }
}

__device__ __forceinline__ void xf_acc(float& S, float& C, float P) {
    const float s = S + P;
    const float bp = s - S;
    const float err = (S - (s - bp)) + (P - bp);
    S = s;
    C += err;
}

template <int DP, int CB, int EXPP>
__global__ void __launch_bounds__(ST)
    kv_xf_sym_kernel(const float2* __restrict__ xs, int64_t n, int nt, float c0,
                     const float* __restrict__ V, int64_t ldv, int ncols,
                     const int4* __restrict__ work, int G, int nchunk,
                     double* __restrict__ prow, double* __restrict__ pcol) {
    extern __shared__ float2 xfsm[];
    float2* sx = xfsm;                                                 // ST * DP
    float* sv = reinterpret_cast<float*>(sx + ST * DP);                // ST * CB
    float (*W)[ST][SCW + 1] = reinterpret_cast<float (*)[ST][SCW + 1]>(sv + ST * CB);
    float2 (*red)[4][SCW] = reinterpret_cast<float2 (*)[4][SCW]>(&W[CB][0][0]);
    const int4 wk = work[blockIdx.x];  // (I, J0, J1, chunk)
    const int I = wk.x;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int64_t i = (int64_t)I * ST + t;
    float2 xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < n) ? xs[i * DP + q] : make_float2(0.f, 0.f);
    float vi[CB], S[CB], C[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        vi[k] = (i < n && k < ncols) ? V[i + (int64_t)k * ldv] : 0.f;
        S[k] = C[k] = 0.f;
    }
    for (int J = wk.y; J < wk.z; ++J) {
        __syncthreads();
        for (int e = t; e < ST * DP; e += ST) {
            const int jj = e / DP;
            const int64_t j = (int64_t)J * ST + jj;
            sx[e] = (j < n) ? xs[j * DP + (e - jj * DP)] : make_float2(0.f, 0.f);
        }
        for (int e = t; e < ST * CB; e += ST) {
            const int k = e / ST, jj = e - k * ST;
            const int64_t j = (int64_t)J * ST + jj;
            sv[jj * CB + k] = (j < n && k < ncols) ? V[j + (int64_t)k * ldv] : 0.f;
        }
        __syncthreads();
        const bool mirror = (J != I);
        for (int cst = 0; cst < ST; cst += SCW) {
            for (int jj = 0; jj < SCW; ++jj) {
                const int jc = cst + jj;
                float a = c0;
#pragma unroll
                for (int q = 0; q < DP; ++q) {
                    const float2 xj = sx[jc * DP + q];
                    const float dl = (xi[q].x - xj.x) + (xi[q].y - xj.y);
                    a = fmaf(-dl, dl, a);
                }
                const float e = xf_exp2<EXPP>(a);
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    xf_acc(S[k], C[k], e * sv[jc * CB + k]);
                    if (mirror) W[k][t][jj] = e * vi[k];
                }
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) df_renorm(S[k], C[k]);
            if (mirror) {
                __syncthreads();
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    float cs = 0.f, cc = 0.f;
                    for (int r = 0; r < 32; ++r) xf_acc(cs, cc, W[k][warp * 32 + r][lane]);
                    red[k][warp][lane] = make_float2(cs, cc);
                }
                __syncthreads();
                if (warp == 0) {
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        double s = 0.0;
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            s += (double)red[k][w][lane].x + (double)red[k][w][lane].y;
                        pcol[(((size_t)J * nt + I) * CB + k) * ST + cst + lane] = s;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CB; ++k)
        prow[(((size_t)I * nchunk + wk.w) * CB + k) * ST + t] = (double)S[k] + (double)C[k];
}

// O = noise V + the partial sums of kv_xf_sym_kernel, in FP64, rounded to FP32.
__global__ void kv_xf_sym_reduce_kernel(const double* __restrict__ prow,
                                        const double* __restrict__ pcol, int nt, int G,
                                        int nchunk, int cb, int ncols,
                                        const float* __restrict__ V, int64_t ldv, float noise,
                                        float* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    const int T = (int)(i / ST), r = (int)(i % ST);
    double s = (double)noise * (double)V[i + (int64_t)k * ldv];
    for (int ch = T / G; ch < nchunk; ++ch) s += prow[(((size_t)T * nchunk + ch) * cb + k) * ST + r];
    for (int I = 0; I < T; ++I) s += pcol[(((size_t)T * nt + I) * cb + k) * ST + r];
    O[i + (int64_t)k * ldo] = (float)s;
}

// ---------------------------------------------------------------------------
// Derivative products dK/dtheta_q W in double-float arithmetic.  The
// gradient's trace term sums w^T (dK r) over a large, rough w = K_y^{-1} r and
// cancels all but ~1e-5 of its magnitude, so the entries K_ij t_ijq^2 need
// about 28 bits even when every rounding is independent per entry (FP32
// entries leave errors of 3e-4 relative on the smaller gradient entries).
// Every quantity is an FP32 pair here: the squared differences from the split
// inputs (exact hi difference, TwoProduct), the exponent summed with TwoSum,
// exp2 of the pair (the table-driven method of kv_df_kernel), the products
// K t^2 and (K t^2) w with TwoProduct, the sums with TwoSum.  Slots as
// dkv_kernel: ARD per dimension then log s^2; isotropic the sum over
// dimensions then log s^2; (x_r - x'_r)^2 / l_r^2 = 2 ln 2 t_r^2 in the exp2
// scaling of x'.
template <int DP, int CB>
__global__ void __launch_bounds__(KT)
    dkv_df_kernel(const float4* __restrict__ xs, int64_t n, int nq, int ard, float c0h,
                  float c0l, const double* __restrict__ W, int64_t ldw, int ncols,
                  const float2* __restrict__ gtab, double* __restrict__ part, int64_t ldp,
                  int64_t cps) {
    __shared__ float2 tab[NTAB];
    __shared__ float4 sx[TJ * DP];
    __shared__ float2 sw[TJ * CB];
    for (int e = threadIdx.x; e < NTAB; e += KT) tab[e] = gtab[e];
    const int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * cps;
    const int64_t j1 = min(n, j0 + cps);
    float4 xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < n) ? xs[i * DP + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    float S[DP + 1][CB], C[DP + 1][CB];
#pragma unroll
    for (int q = 0; q <= DP; ++q)
#pragma unroll
        for (int k = 0; k < CB; ++k) S[q][k] = C[q][k] = 0.f;
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        const int jn = (int)min((int64_t)TJ, j1 - jt);
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DP; e += KT) {
            const int jj = e / DP;
            sx[e] = (jj < jn) ? xs[(jt + jj) * DP + (e - jj * DP)] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = threadIdx.x; e < TJ * CB; e += KT) {
            const int k = e / TJ, jj = e - k * TJ;
            const double w = (jj < jn && k < ncols) ? W[(jt + jj) + (int64_t)k * ldw] : 0.0;
            const float wh = (float)w;
            sw[jj * CB + k] = make_float2(wh, (float)(w - (double)wh));
        }
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            float Ph[DP], Pl[DP];  // t_q^2 as pairs
            float ah = c0h, al = c0l;
#pragma unroll
            for (int q = 0; q < DP; ++q) {
                const float4 xj = sx[jj * DP + q];
                const float D = xi[q].x - xj.x;  // exact
                const float E = (xi[q].y - xj.y) + (xi[q].z - xj.z);
                const float P = D * D;
                float Pe = fmaf(D, D, -P);
                Pe = fmaf(D, E + E, Pe);
                Pe = fmaf(E, E, Pe);
                Ph[q] = P;
                Pl[q] = Pe;
                df_sub(ah, al, P, Pe);
            }
            const DF e = df_exp2(ah, al, tab);
#pragma unroll
            for (int q = 0; q <= DP; ++q) {
                float uh, ul;  // e * t_q^2 (or e itself for log s^2)
                if (q < DP) {
                    uh = e.h * Ph[q];
                    ul = fmaf(e.h, Ph[q], -uh);
                    ul = fmaf(e.h, Pl[q], ul);
                    ul = fmaf(e.l, Ph[q], ul);
                } else {
                    uh = e.h;
                    ul = e.l;
                }
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const float2 w = sw[jj * CB + k];
                    const float ph = uh * w.x;
                    float pl = fmaf(uh, w.x, -ph);
                    pl = fmaf(uh, w.y, pl);
                    pl = fmaf(ul, w.x, pl);
                    df_acc(S[q][k], C[q][k], ph, pl);
                }
            }
            if ((jj & 31) == 31)
#pragma unroll
                for (int q = 0; q <= DP; ++q)
#pragma unroll
                    for (int k = 0; k < CB; ++k) df_renorm(S[q][k], C[q][k]);
        }
    }
    if (i >= n) return;
    constexpr double kScale = 1.3862943611198906;  // 2 ln 2
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        if (k >= ncols) break;
        double* base = part + ((int64_t)blockIdx.y * CB + k) * (int64_t)nq * ldp;
        if (ard) {
#pragma unroll
            for (int q = 0; q < DP; ++q)
                if (q < nq - 1)
                    base[(int64_t)q * ldp + i] = kScale * ((double)S[q][k] + (double)C[q][k]);
        } else {
            double sum = 0.0;
#pragma unroll
            for (int q = 0; q < DP; ++q) sum += (double)S[q][k] + (double)C[q][k];
            base[i] = kScale * sum;
        }
        base[(int64_t)(nq - 1) * ldp + i] = (double)S[DP][k] + (double)C[DP][k];
    }
}

__global__ void dkv_df_reduce_kernel(const double* __restrict__ part, int64_t ldp, int nsplit,
                                     int cb, int nq, int ncols, double* __restrict__ G,
                                     int64_t ldg, int64_t c_total, int k0, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y, k = blockIdx.z;
    if (i >= n || k >= ncols) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[(((int64_t)sp * cb + k) * nq + q) * ldp + i];
    G[(int64_t)q * ldg * c_total + (int64_t)(k0 + k) * ldg + i] = s;
}

__global__ void kv_df_sym_reduce_kernel(const double* __restrict__ prow,
                                        const double* __restrict__ pcol, int nt, int G,
                                        int nchunk, int cb, int ncols,
                                        const double* __restrict__ V, int64_t ldv, double noise,
                                        const double* __restrict__ B, int64_t ldb,
                                        double* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    const int T = (int)(i / ST), r = (int)(i % ST);
    double s = noise * V[i + (int64_t)k * ldv];
    for (int ch = T / G; ch < nchunk; ++ch) s += prow[(((size_t)T * nchunk + ch) * cb + k) * ST + r];
    for (int I = 0; I < T; ++I) s += pcol[(((size_t)T * nt + I) * cb + k) * ST + r];
    O[i + (int64_t)k * ldo] = B ? (B[i + (int64_t)k * ldb] - s) : s;
}

__global__ void kv_df_reduce_kernel(const double* __restrict__ part, int64_t ldp, int nsplit,
                                    int cb, int ncols, const double* __restrict__ V, int64_t ldv,
                                    double noise, const double* __restrict__ B, int64_t ldb,
                                    double* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    double s = noise * V[i + (int64_t)k * ldv];
    for (int sp = 0; sp < nsplit; ++sp) s += part[((int64_t)sp * cb + k) * ldp + i];
    O[i + (int64_t)k * ldo] = B ? (B[i + (int64_t)k * ldb] - s) : s;
}

// Column-wise max |x'| (FP64) to pick the grid of the hi parts.
__global__ void colmax_kernel(const double* __restrict__ xs64, int64_t n, int dp,
                              double* __restrict__ out) {
    __shared__ double sh[256];
    const int q = blockIdx.x;
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(xs64[i * dp + q]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

// hi = x' rounded to the grid 2^(k_r - 23), lo = fl(x' - hi), lo2 = x' - hi - lo.
// The (hi, lo) pairs alone feed the exact-difference FP32 kernel.
__global__ void df_prep_kernel(const double* __restrict__ xs64, int64_t n, int dp, double scale,
                               const double* __restrict__ grid, float4* __restrict__ out,
                               float2* __restrict__ out2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * dp) return;
    const int q = (int)(e % dp);
    const double x = xs64[e] * scale;
    const double g = grid[q];
    const double hi = rint(x / g) * g;
    const float lo = (float)(x - hi);
    const float lo2 = (float)(x - hi - (double)lo);
    out[e] = make_float4((float)hi, lo, lo2, 0.f);
    out2[e] = make_float2((float)hi, lo);
}

struct DfSplit {
    int nrb, nsplit;
    int64_t cps, ldp;
};

DfSplit df_plan(int64_t n) {
    DfSplit s;
    s.nrb = (int)((n + KT - 1) / KT);
    const int64_t target = (int64_t)sm_count_df() * 8;
    int64_t ns = (target + s.nrb - 1) / s.nrb;
    ns = std::max<int64_t>(1, std::min(ns, (n + TJ - 1) / TJ));
    int64_t cps = (n + ns - 1) / ns;
    cps = ((cps + TJ - 1) / TJ) * TJ;
    s.cps = cps;
    s.nsplit = (int)((n + cps - 1) / cps);
    s.ldp = ((n + 31) / 32) * 32;
    return s;
}

template <int DP, int CB>
void df_launch(const float4* xs, int64_t n, float c0h, float c0l, const double* V, int64_t ldv,
               int ncols, const float2* tab, double* part, const DfSplit& s, cudaStream_t st) {
    kv_df_kernel<DP, CB><<<dim3(s.nrb, s.nsplit), KT, 0, st>>>(xs, n, c0h, c0l, V, ldv, ncols,
                                                               tab, part, s.ldp, s.cps);
    KPCG_LAUNCHED("kv_df_kernel");
}

template <int DP>
void df_launch_cb(int cb, const float4* xs, int64_t n, float c0h, float c0l, const double* V,
                  int64_t ldv, int ncols, const float2* tab, double* part, const DfSplit& s,
                  cudaStream_t st) {
    switch (cb) {
        case 1: df_launch<DP, 1>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st); break;
        case 2: df_launch<DP, 2>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st); break;
        case 4: df_launch<DP, 4>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st); break;
        case 8:
            if constexpr (DP <= 16) {
                df_launch<DP, 8>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st);
                break;
            }
            fail(KPCG_ERR_ARG, "internal: bad column block");
        case 16:
            if constexpr (DP <= 12) {
                df_launch<DP, 16>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st);
                break;
            }
            fail(KPCG_ERR_ARG, "internal: bad column block");
        default: fail(KPCG_ERR_ARG, "internal: bad column block");
    }
}

// Widest column block of the plain kernel for a padded dimension (registers).
static int df_max_cb(int dp) { return dp <= 12 ? 16 : dp <= 16 ? 8 : 4; }

// Column blocks of a product: greedy widest-first, then the smallest block
// (of the allowed widths) that holds the remainder.
static std::vector<int> df_blocks(int c, int maxcb) {
    std::vector<int> out;
    while (c > 0) {
        int cb = maxcb;
        while (cb > 1 && cb / 2 >= c) cb /= 2;
        out.push_back(cb);
        c -= std::min(cb, c);
    }
    return out;
}

// FP32-pipe instructions per product (the model of the benchmark): the
// symmetric kernel evaluates n(n+1)/2 entries per pass of <= 2 columns and
// spends 24 per entry and column (row and mirrored column), the plain one n^2
// entries per pass and 12 per entry and column.
static bool df_prefer_plain(int64_t n, int dp, int c) {
    const double e = 16.0 * dp + 33.0;
    double sym = 0.0, plain = 0.0;
    for (int k = 0; k < c; k += 2) sym += 0.5 * (e + 24.0 * std::min(2, c - k));
    for (int cb : df_blocks(c, df_max_cb(dp))) plain += e + 12.0 * cb;
    (void)n;
    return plain < sym;
}

}  // namespace

// Refresh the double-float inputs of the handle after theta changed.
void df_prepare(Ctx& h) {
    if (h.df_version == h.theta_version) return;
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    if (!h.df_tab.p) {
        std::vector<float2> t(NTAB);
        for (int j = -128; j <= 128; ++j) {
            const double v = std::exp2((double)j / 256.0);
            const float hi = (float)v;
            t[j + 128] = make_float2(hi, (float)(v - (double)hi));
        }
        h.df_tab.need(NTAB);
        KPCG_CUDA(cudaMemcpyAsync(h.df_tab.p, t.data(), sizeof(float2) * NTAB,
                                  cudaMemcpyHostToDevice, st));
        std::vector<float2> t1(NTAB1K);
        for (int j = 0; j < NTAB1K; ++j) {
            const double v = std::exp2((double)j / NTAB1K);
            const float hi = (float)v;
            t1[j] = make_float2(hi, (float)(v - (double)hi));
        }
        h.df_tab1k.need(NTAB1K);
        KPCG_CUDA(cudaMemcpyAsync(h.df_tab1k.p, t1.data(), sizeof(float2) * NTAB1K,
                                  cudaMemcpyHostToDevice, st));
        KPCG_CUDA(cudaStreamSynchronize(st));  // the host tables leave scope
    }
    // x' in the exp2 scaling: xs64 * sqrt(log2 e)
    const double scale = std::sqrt(kLog2e);
    double* mx = h.df_grid.need((size_t)2 * h.dp);
    colmax_kernel<<<h.dp, 256, 0, st>>>(h.xs64.p, n, h.dp, mx);
    KPCG_LAUNCHED("colmax_kernel");
    std::vector<double> hm((size_t)h.dp), grid((size_t)h.dp);
    KPCG_CUDA(cudaMemcpyAsync(hm.data(), mx, sizeof(double) * h.dp, cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < h.dp; ++q) {
        const double m = hm[q] * scale;
        int k = 0;
        if (m > 0.0) k = (int)std::floor(std::log2(m)) + 1;  // |x'| < 2^k
        grid[q] = std::ldexp(1.0, k - 23);
    }
    KPCG_CUDA(cudaMemcpyAsync(mx + h.dp, grid.data(), sizeof(double) * h.dp,
                              cudaMemcpyHostToDevice, st));
    float4* xdf = reinterpret_cast<float4*>(h.xdf.need((size_t)n * h.dp * 4));
    float2* xf2 = reinterpret_cast<float2*>(h.xf2.need((size_t)n * h.dp * 2));
    df_prep_kernel<<<(unsigned)((n * h.dp + 255) / 256), 256, 0, st>>>(h.xs64.p, n, h.dp, scale,
                                                                       mx + h.dp, xdf, xf2);
    KPCG_LAUNCHED("df_prep_kernel");
    const double c0 = std::log2(h.s2);
    h.df_c0h = (float)c0;
    h.df_c0l = (float)(c0 - (double)h.df_c0h);
    h.df_version = h.theta_version;
}

template <int DP, int CB>
static size_t df_sym_smem() {
    return sizeof(float4) * ST * DP + sizeof(float2) * (NTAB + 1) + sizeof(float2) * ST * CB +
           sizeof(float2) * CB * ST * (SCW + 1) + sizeof(float2) * CB * 4 * SCW;
}

template <int DP, int CB>
static void df_sym_launch1(const float4* xs, int64_t n, int nt, float c0h, float c0l,
                           const double* V, int64_t ldv, int ncols, const float2* tab,
                           const int4* work, int nwork, int G, int nchunk, double* prow,
                           double* pcol, cudaStream_t st) {
    const size_t smem = df_sym_smem<DP, CB>();
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_df_sym_kernel<DP, CB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    kv_df_sym_kernel<DP, CB><<<nwork, ST, smem, st>>>(xs, n, nt, c0h, c0l, V, ldv, ncols, tab,
                                                      work, G, nchunk, prow, pcol);
    KPCG_LAUNCHED("kv_df_sym_kernel");
}

template <int DP>
static void df_sym_launch(int cb, const float4* xs, int64_t n, int nt, float c0h, float c0l,
                          const double* V, int64_t ldv, int ncols, const float2* tab,
                          const int4* work, int nwork, int G, int nchunk, double* prow,
                          double* pcol, cudaStream_t st) {
    if (cb == 1)
        df_sym_launch1<DP, 1>(xs, n, nt, c0h, c0l, V, ldv, ncols, tab, work, nwork, G, nchunk,
                              prow, pcol, st);
    else
        df_sym_launch1<DP, 2>(xs, n, nt, c0h, c0l, V, ldv, ncols, tab, work, nwork, G, nchunk,
                              prow, pcol, st);
}

// Symmetric product, column blocks of two.  Work items (I, J0, J1, chunk) cover
// the upper triangle of tile pairs in runs of G tiles, cached per n.
// Work list (I, J0, J1, chunk) over the upper triangle of tile pairs, in runs
// of G tiles, cached per n.  Returns G; nchunk = ceil(nt / G).
static int ensure_sym_work(Ctx& h, int nt) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    // runs of G tiles: about sixteen CTAs of work per SM
    int G = std::max(1, (int)((int64_t)nt * (nt + 1) / 2 / ((int64_t)sm_count_df() * 16)));
    G = std::min(G, 16);
    if (h.df_sym_n != n || h.df_sym_G != G) {
        std::vector<int4> w;
        for (int I = 0; I < nt; ++I)
            for (int J0 = I; J0 < nt;) {
                const int ch = J0 / G;
                const int J1 = std::min(nt, (ch + 1) * G);
                w.push_back(make_int4(I, J0, J1, ch));
                J0 = J1;
            }
        int4* dw = reinterpret_cast<int4*>(h.df_work.need(w.size() * 4));
        KPCG_CUDA(cudaMemcpyAsync(dw, w.data(), sizeof(int4) * w.size(), cudaMemcpyHostToDevice,
                                  st));
        KPCG_CUDA(cudaStreamSynchronize(st));
        h.df_sym_n = n;
        h.df_sym_G = G;
        h.df_nwork = (int)w.size();
    }
    return G;
}

static void kv_df_sym(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb,
                      double* O, int64_t ldo, double noise) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int nt = (int)((n + ST - 1) / ST);
    const int G = ensure_sym_work(h, nt);
    const int nchunk = (nt + G - 1) / G;
    const int max_cb = 2;
    double* prow = h.df_prow.need((size_t)nt * nchunk * max_cb * ST);
    double* pcol = h.df_pcol.need((size_t)nt * nt * max_cb * ST);
    const float4* xs = reinterpret_cast<const float4*>(h.xdf.p);
    const float2* tab = reinterpret_cast<const float2*>(h.df_tab.p);
    const int4* work = reinterpret_cast<const int4*>(h.df_work.p);
    for (int k0 = 0; k0 < c;) {
        const int cb = (c - k0 >= 2) ? 2 : 1;
        const int ncols = cb;
        const double* Vk = V + (int64_t)k0 * ldv;
        switch (h.dp) {
            case 4: df_sym_launch<4>(cb, xs, n, nt, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            case 8: df_sym_launch<8>(cb, xs, n, nt, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            case 12: df_sym_launch<12>(cb, xs, n, nt, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            case 16: df_sym_launch<16>(cb, xs, n, nt, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        kv_df_sym_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            prow, pcol, nt, G, nchunk, cb, ncols, Vk, ldv, noise,
            B ? B + (int64_t)k0 * ldb : nullptr, ldb, O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("kv_df_sym_reduce_kernel");
        k0 += ncols;
    }
}

template <int DP, int CB>
static void f64_sym_launch1(const double* xs, int64_t n, int nt, double c0, const double* V,
                            int64_t ldv, int ncols, const int4* work, int nwork, int G, int nchunk,
                            double* prow, double* pcol, const double* tab64, cudaStream_t st) {
    const size_t smem =
        sizeof(double) * (ST * DP + ST * CB + CB * ST * (SCW + 1) + CB * 4 * SCW + NTAB64);
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_f64_sym_kernel<DP, CB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    kv_f64_sym_kernel<DP, CB><<<nwork, ST, smem, st>>>(xs, n, nt, c0, V, ldv, ncols, work, G,
                                                       nchunk, prow, pcol, tab64);
    KPCG_LAUNCHED("kv_f64_sym_kernel");
}

template <int DP>
static void f64_sym_launch(int cb, const double* xs, int64_t n, int nt, double c0, const double* V,
                           int64_t ldv, int ncols, const int4* work, int nwork, int G, int nchunk,
                           double* prow, double* pcol, const double* tab64, cudaStream_t st) {
    if (cb == 1)
        f64_sym_launch1<DP, 1>(xs, n, nt, c0, V, ldv, ncols, work, nwork, G, nchunk, prow, pcol, tab64, st);
    else
        f64_sym_launch1<DP, 2>(xs, n, nt, c0, V, ldv, ncols, work, nwork, G, nchunk, prow, pcol, tab64, st);
}

void kv_f64_sym(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb,
                double* O, int64_t ldo, double noise) {
    if (h.n <= 0 || c <= 0) return;
    if (!(h.dp <= 16 && h.n >= 4 * ST)) {
        kv_f64(h.xs64.p, h.n, h.dp, h.c0_64(), noise, V, ldv, c, B, ldb, O, ldo, h.kvws, h.stream);
        return;
    }
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int nt = (int)((n + ST - 1) / ST);
    const int G = ensure_sym_work(h, nt);
    const int nchunk = (nt + G - 1) / G;
    const int max_cb = 2;
    double* prow = h.df_prow.need((size_t)nt * nchunk * max_cb * ST);
    double* pcol = h.df_pcol.need((size_t)nt * nt * max_cb * ST);
    const int4* work = reinterpret_cast<const int4*>(h.df_work.p);
    const double c0 = h.c0_64();
    if (!h.f64_tab.p) {
        std::vector<double> t(NTAB64);
        for (int j = 0; j < NTAB64; ++j) t[j] = std::exp2((double)j / NTAB64);
        h.f64_tab.need(NTAB64);
        KPCG_CUDA(cudaMemcpyAsync(h.f64_tab.p, t.data(), sizeof(double) * NTAB64,
                                  cudaMemcpyHostToDevice, st));
        KPCG_CUDA(cudaStreamSynchronize(st));
    }
    const double* tab64 = h.f64_tab.p;
    for (int k0 = 0; k0 < c;) {
        const int cb = (c - k0 >= 2) ? 2 : 1;
        const double* Vk = V + (int64_t)k0 * ldv;
        switch (h.dp) {
            case 4: f64_sym_launch<4>(cb, h.xs64.p, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, tab64, st); break;
            case 8: f64_sym_launch<8>(cb, h.xs64.p, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, tab64, st); break;
            case 12: f64_sym_launch<12>(cb, h.xs64.p, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, tab64, st); break;
            case 16: f64_sym_launch<16>(cb, h.xs64.p, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, tab64, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        kv_df_sym_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)cb), 256, 0, st>>>(
            prow, pcol, nt, G, nchunk, cb, cb, Vk, ldv, noise, B ? B + (int64_t)k0 * ldb : nullptr,
            ldb, O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("kv_df_sym_reduce_kernel");
        k0 += cb;
    }
}

void kv_df(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb, double* O,
           int64_t ldo, double noise) {
    if (h.n <= 0 || c <= 0) return;
    // the squared distances on the tensor cores where the sliced layout fits
    if (h.df_tensor && kv_tcd_supported(h)) {
        kv_tcd(h, V, ldv, c, B, ldb, O, ldo, noise);
        return;
    }
    df_prepare(h);
    // The symmetric kernel pays off once there are several tile pairs per SM,
    // and while few columns are in the product.
    if (h.dp <= 16 && h.n >= 4 * ST && h.df_symmetric && !df_prefer_plain(h.n, h.dp, c)) {
        kv_df_sym(h, V, ldv, c, B, ldb, O, ldo, noise);
        return;
    }
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const DfSplit s = df_plan(n);
    const int max_cb = df_max_cb(h.dp);
    double* part = h.kvws.part64.need((size_t)s.nsplit * max_cb * s.ldp);
    const float4* xs = reinterpret_cast<const float4*>(h.xdf.p);
    const float2* tab = reinterpret_cast<const float2*>(h.df_tab.p);
    const std::vector<int> blocks = df_blocks(c, max_cb);
    int k0 = 0;
    for (int cb : blocks) {
        const int ncols = std::min(cb, c - k0);
        const double* Vk = V + (int64_t)k0 * ldv;
        switch (h.dp) {
            case 4: df_launch_cb<4>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 8: df_launch_cb<8>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 12: df_launch_cb<12>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 16: df_launch_cb<16>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 32: df_launch_cb<32>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        kv_df_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            part, s.ldp, s.nsplit, cb, ncols, Vk, ldv, noise, B ? B + (int64_t)k0 * ldb : nullptr,
            ldb, O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("kv_df_reduce_kernel");
        k0 += ncols;
    }
}

template <int DP, int CB, int EXPP>
static void xf_sym_launch1(const float2* xs, int64_t n, int nt, float c0, const float* V,
                           int64_t ldv, int ncols, const int4* work, int nwork, int G, int nchunk,
                           double* prow, double* pcol, cudaStream_t st) {
    const size_t smem = sizeof(float2) * ST * DP + sizeof(float) * ST * CB +
                        sizeof(float) * CB * ST * (SCW + 1) + sizeof(float2) * CB * 4 * SCW;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_xf_sym_kernel<DP, CB, EXPP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    kv_xf_sym_kernel<DP, CB, EXPP><<<nwork, ST, smem, st>>>(xs, n, nt, c0, V, ldv, ncols, work, G,
                                                            nchunk, prow, pcol);
    KPCG_LAUNCHED("kv_xf_sym_kernel");
}

template <int DP>
static void xf_sym_launch(int cb, int expp, const float2* xs, int64_t n, int nt, float c0,
                          const float* V, int64_t ldv, int ncols, const int4* work, int nwork,
                          int G, int nchunk, double* prow, double* pcol, cudaStream_t st) {
    if (expp == 0) {
        if (cb == 1)
            xf_sym_launch1<DP, 1, 0>(xs, n, nt, c0, V, ldv, ncols, work, nwork, G, nchunk, prow, pcol, st);
        else
            xf_sym_launch1<DP, 2, 0>(xs, n, nt, c0, V, ldv, ncols, work, nwork, G, nchunk, prow, pcol, st);
    } else {
        if (cb == 1)
            xf_sym_launch1<DP, 1, 1>(xs, n, nt, c0, V, ldv, ncols, work, nwork, G, nchunk, prow, pcol, st);
        else
            xf_sym_launch1<DP, 2, 1>(xs, n, nt, c0, V, ldv, ncols, work, nwork, G, nchunk, prow, pcol, st);
    }
}

bool kv_xf_supported(const Ctx& h) { return h.dp <= 16 && h.n >= 1; }

void kv_xf(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo, float noise,
           int expp) {
    if (h.n <= 0 || c <= 0) return;
    if (!kv_xf_supported(h)) fail(KPCG_ERR_ARG, "exact-difference FP32 K.V needs d <= 16");
    df_prepare(h);
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int nt = (int)((n + ST - 1) / ST);
    const int G = ensure_sym_work(h, nt);
    const int nchunk = (nt + G - 1) / G;
    const int max_cb = 2;
    double* prow = h.df_prow.need((size_t)nt * nchunk * max_cb * ST);
    double* pcol = h.df_pcol.need((size_t)nt * nt * max_cb * ST);
    const float2* xs = reinterpret_cast<const float2*>(h.xf2.p);
    const int4* work = reinterpret_cast<const int4*>(h.df_work.p);
    const float c0 = h.df_c0h;
    for (int k0 = 0; k0 < c;) {
        const int cb = (c - k0 >= 2) ? 2 : 1;
        const float* Vk = V + (int64_t)k0 * ldv;
        switch (h.dp) {
            case 4: xf_sym_launch<4>(cb, expp, xs, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            case 8: xf_sym_launch<8>(cb, expp, xs, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            case 12: xf_sym_launch<12>(cb, expp, xs, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            case 16: xf_sym_launch<16>(cb, expp, xs, n, nt, c0, Vk, ldv, cb, work, h.df_nwork, G, nchunk, prow, pcol, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        kv_xf_sym_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)cb), 256, 0, st>>>(
            prow, pcol, nt, G, nchunk, cb, cb, Vk, ldv, noise, O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("kv_xf_sym_reduce_kernel");
        k0 += cb;
    }
}

template <int DP, int CB>
static void dkv_df_launch1(const float4* xs, int64_t n, int nq, int ard, float c0h, float c0l,
                           const double* W, int64_t ldw, int ncols, const float2* tab,
                           double* part, const DfSplit& s, cudaStream_t st) {
    dkv_df_kernel<DP, CB><<<dim3(s.nrb, s.nsplit), KT, 0, st>>>(xs, n, nq, ard, c0h, c0l, W, ldw,
                                                               ncols, tab, part, s.ldp, s.cps);
    KPCG_LAUNCHED("dkv_df_kernel");
}

void dkv_df(Ctx& h, const double* W, int64_t ldw, int c, double* G, int64_t ldg) {
    if (h.n <= 0 || c <= 0) return;
    if (h.dp > 16) fail(KPCG_ERR_ARG, "double-float derivative products need d <= 16");
    df_prepare(h);
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int nq = (h.ard ? h.d : 1) + 1;
    const DfSplit s = df_plan(n);
    const int max_cb = h.dp <= 8 ? 2 : 1;
    double* part = h.kvws.part64.need((size_t)s.nsplit * max_cb * nq * s.ldp);
    const float4* xs = reinterpret_cast<const float4*>(h.xdf.p);
    const float2* tab = reinterpret_cast<const float2*>(h.df_tab.p);
    for (int k0 = 0; k0 < c;) {
        const int cb = std::min(max_cb, c - k0);
        const double* Wk = W + (int64_t)k0 * ldw;
#define KPCG_DKVDF(DPV)                                                                        \
    case DPV:                                                                                  \
        if (cb == 1)                                                                           \
            dkv_df_launch1<DPV, 1>(xs, n, nq, h.ard, h.df_c0h, h.df_c0l, Wk, ldw, cb, tab, part, \
                                   s, st);                                                     \
        else if constexpr (DPV <= 8)                                                           \
            dkv_df_launch1<DPV, 2>(xs, n, nq, h.ard, h.df_c0h, h.df_c0l, Wk, ldw, cb, tab, part, \
                                   s, st);                                                     \
        break;
        switch (h.dp) {
            KPCG_DKVDF(4)
            KPCG_DKVDF(8)
            KPCG_DKVDF(12)
            KPCG_DKVDF(16)
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
#undef KPCG_DKVDF
        dim3 rg((unsigned)((n + 255) / 256), (unsigned)nq, (unsigned)cb);
        dkv_df_reduce_kernel<<<rg, 256, 0, st>>>(part, s.ldp, s.nsplit, cb, nq, cb, G, ldg, c, k0,
                                                 n);
        KPCG_LAUNCHED("dkv_df_reduce_kernel");
        k0 += cb;
    }
}

}  // namespace kpcg
