// Matrix-free kernel products on the CUDA cores.
//
// The only operation CG needs from K_y is a product with a block of vectors
// (Sec. 2.1); entries are rebuilt from X for every product, so nothing n x n
// is stored (storing K on the fly is named as the way to scale in Sec. 6).
// Entries follow Eq. 1 by DIRECT DIFFERENCES on pre-scaled inputs x'
// (no norm expansion), so these kernels are the accurate references of the
// GPU path: FP64 for the outer residual of the refinement and the FP64 solver,
// FP32 for the plain-FP32 baseline solver.
//
// Work split: a CTA owns KT*RPT rows (one or two per thread, x_i in
// registers) and a contiguous range of columns j; column tiles of x_j and V_j
// are staged in shared memory and broadcast to all threads.  Column ranges
// write separate partial sums that a second kernel adds in a fixed order
// (deterministic; no atomics).
#include <cuda_runtime.h>

#include <algorithm>

#include "kpcg_internal.cuh"

namespace kpcg {
namespace {

template <typename T>
__device__ __forceinline__ T kexp(T a);
template <>
__device__ __forceinline__ float kexp<float>(float a) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}
template <>
__device__ __forceinline__ double kexp<double>(double a) {
    return exp(a);
}

constexpr int KT = 256;  // threads per CTA
constexpr int TJ = 64;   // columns per shared-memory tile

int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        if (cached <= 0) cached = 148;
    }
    return cached;
}

template <typename T, int DP, int CB, int RPT>
__global__ void __launch_bounds__(KT)
    kv_simt_kernel(const T* __restrict__ xs, int64_t n, T c0, const T* __restrict__ V,
                   int64_t ldv, int ncols, T* __restrict__ part, int64_t ldp, int64_t cps) {
    __shared__ __align__(16) T sx[TJ * DP];
    __shared__ __align__(16) T sv[TJ * CB];
    const int64_t rbase = (int64_t)blockIdx.x * (KT * RPT) + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * cps;
    const int64_t j1 = min(n, j0 + cps);
    T xi[RPT][DP];
    T acc[RPT][CB];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t i = rbase + (int64_t)r * KT;
#pragma unroll
        for (int q = 0; q < DP; ++q) xi[r][q] = (i < n) ? xs[i * DP + q] : T(0);
#pragma unroll
        for (int k = 0; k < CB; ++k) acc[r][k] = T(0);
    }
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        const int jn = (int)min((int64_t)TJ, j1 - jt);
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DP; e += KT) {
            const int jj = e / DP;
            sx[e] = (jj < jn) ? xs[(jt + jj) * DP + (e - jj * DP)] : T(0);
        }
        for (int e = threadIdx.x; e < TJ * CB; e += KT) {
            const int k = e / TJ, jj = e - k * TJ;
            sv[jj * CB + k] = (jj < jn && k < ncols) ? V[(jt + jj) + (int64_t)k * ldv] : T(0);
        }
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            T xj[DP], vj[CB];
#pragma unroll
            for (int q = 0; q < DP; ++q) xj[q] = sx[jj * DP + q];
#pragma unroll
            for (int k = 0; k < CB; ++k) vj[k] = sv[jj * CB + k];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                T a = c0;
#pragma unroll
                for (int q = 0; q < DP; ++q) {
                    const T t = xi[r][q] - xj[q];
                    a = fma(-t, t, a);
                }
                const T e = kexp<T>(a);
#pragma unroll
                for (int k = 0; k < CB; ++k) acc[r][k] = fma(e, vj[k], acc[r][k]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t i = rbase + (int64_t)r * KT;
        if (i < n) {
#pragma unroll
            for (int k = 0; k < CB; ++k)
                if (k < ncols) part[((int64_t)blockIdx.y * CB + k) * ldp + i] = acc[r][k];
        }
    }
}

// O = sum_s part_s + noise V   (or B - that when B is given).
template <typename T>
__global__ void kv_reduce_kernel(const T* __restrict__ part, int64_t ldp, int nsplit, int cb,
                                 int ncols, const T* __restrict__ V, int64_t ldv, T noise,
                                 const T* __restrict__ B, int64_t ldb, T* __restrict__ O,
                                 int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    T s = noise * V[i + (int64_t)k * ldv];
    for (int sp = 0; sp < nsplit; ++sp) s += part[((int64_t)sp * cb + k) * ldp + i];
    O[i + (int64_t)k * ldo] = B ? (B[i + (int64_t)k * ldb] - s) : s;
}

struct Split {
    int nrb, nsplit;
    int64_t cps, ldp;
};

Split plan(int64_t n, int rows_per_cta) {
    Split s;
    s.nrb = (int)((n + rows_per_cta - 1) / rows_per_cta);
    const int64_t target = (int64_t)sm_count() * 8;
    int64_t ns = (target + s.nrb - 1) / s.nrb;
    const int64_t max_ns = (n + TJ - 1) / TJ;
    ns = std::max<int64_t>(1, std::min(ns, max_ns));
    int64_t cps = (n + ns - 1) / ns;
    cps = ((cps + TJ - 1) / TJ) * TJ;
    s.cps = cps;
    s.nsplit = (int)((n + cps - 1) / cps);
    s.ldp = ((n + 31) / 32) * 32;
    return s;
}

template <typename T, int DP, int CB>
void launch_chunk(const T* xs, int64_t n, T c0, const T* V, int64_t ldv, int ncols, T* part,
                  const Split& s, int rpt, cudaStream_t st) {
    dim3 grid(s.nrb, s.nsplit);
    if (rpt == 2)
        kv_simt_kernel<T, DP, CB, 2><<<grid, KT, 0, st>>>(xs, n, c0, V, ldv, ncols, part, s.ldp,
                                                          s.cps);
    else
        kv_simt_kernel<T, DP, CB, 1><<<grid, KT, 0, st>>>(xs, n, c0, V, ldv, ncols, part, s.ldp,
                                                          s.cps);
    KPCG_LAUNCHED("kv_simt_kernel");
}

template <typename T, int DP>
void launch_cb(int cb, const T* xs, int64_t n, T c0, const T* V, int64_t ldv, int ncols, T* part,
               const Split& s, int rpt, cudaStream_t st) {
    switch (cb) {
        case 1: launch_chunk<T, DP, 1>(xs, n, c0, V, ldv, ncols, part, s, rpt, st); break;
        case 2: launch_chunk<T, DP, 2>(xs, n, c0, V, ldv, ncols, part, s, rpt, st); break;
        case 4: launch_chunk<T, DP, 4>(xs, n, c0, V, ldv, ncols, part, s, rpt, st); break;
        case 8: launch_chunk<T, DP, 8>(xs, n, c0, V, ldv, ncols, part, s, rpt, st); break;
        case 16:
            // FP64 only (one pass over up to 16 columns: the FP64 exp is the
            // expensive part of an entry, so it is computed once per entry)
            if constexpr (sizeof(T) == 8 && DP <= 16) {
                launch_chunk<T, DP, 16>(xs, n, c0, V, ldv, ncols, part, s, rpt, st);
                break;
            }
            fail(KPCG_ERR_ARG, "internal: bad column block");
        default: fail(KPCG_ERR_ARG, "internal: bad column block");
    }
}

template <typename T>
void kv_generic(const T* xs, int64_t n, int dp, T c0, T noise, const T* V, int64_t ldv, int c,
                const T* B, int64_t ldb, T* O, int64_t ldo, DevBuf<T>& partbuf,
                cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    // Two rows per thread where registers allow (FP32, d <= 16).
    const int rpt = (sizeof(T) == 4 && dp <= 16) ? 2 : 1;
    const Split s = plan(n, KT * rpt);
    const int max_cb = (sizeof(T) == 8 && dp <= 16) ? 16 : 8;
    T* part = partbuf.need((size_t)s.nsplit * max_cb * s.ldp);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = (rem > 8 && max_cb == 16) ? 16 : rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        const T* Vk = V + (int64_t)k0 * ldv;
        switch (dp) {
            case 4: launch_cb<T, 4>(cb, xs, n, c0, Vk, ldv, ncols, part, s, rpt, st); break;
            case 8: launch_cb<T, 8>(cb, xs, n, c0, Vk, ldv, ncols, part, s, rpt, st); break;
            case 12: launch_cb<T, 12>(cb, xs, n, c0, Vk, ldv, ncols, part, s, rpt, st); break;
            case 16: launch_cb<T, 16>(cb, xs, n, c0, Vk, ldv, ncols, part, s, rpt, st); break;
            case 32: launch_cb<T, 32>(cb, xs, n, c0, Vk, ldv, ncols, part, s, rpt, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        dim3 rg((unsigned)((n + 255) / 256), (unsigned)ncols);
        kv_reduce_kernel<T><<<rg, 256, 0, st>>>(part, s.ldp, s.nsplit, cb, ncols, Vk, ldv, noise,
                                                B ? B + (int64_t)k0 * ldb : nullptr, ldb,
                                                O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("kv_reduce_kernel");
        k0 += ncols;
    }
}

// ------------------------------------------------------------ K(X, U) blocks
__global__ void kxu_f32_kernel(const float* __restrict__ xs, int64_t n,
                               const float* __restrict__ us, int64_t m, int dp, float c0,
                               float* __restrict__ KXU) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const int64_t i = e / m, a = e - i * m;
    float acc = c0;
    for (int q = 0; q < dp; ++q) {
        const float t = xs[i * dp + q] - us[a * dp + q];
        acc = fmaf(-t, t, acc);
    }
    KXU[e] = kexp<float>(acc);
}

__global__ void kxu_pair_kernel(const double* __restrict__ xs, int64_t n,
                                const double* __restrict__ us, int64_t m, int dp, double c0,
                                float2* __restrict__ KXU) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    const int64_t i = e / m, a = e - i * m;
    double acc = c0;
    for (int q = 0; q < dp; ++q) {
        const double t = xs[i * dp + q] - us[a * dp + q];
        acc = fma(-t, t, acc);
    }
    const double v = exp(acc);
    const float hi = (float)v;
    KXU[e] = make_float2(hi, (float)(v - (double)hi));
}

__global__ void kuu_f64_kernel(const double* __restrict__ us, int64_t m, int dp, double c0,
                               double scale, double diag_add, double* __restrict__ A) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int64_t a = e / m, b = e - a * m;
    double acc = c0;
    for (int q = 0; q < dp; ++q) {
        const double t = us[a * dp + q] - us[b * dp + q];
        acc = fma(-t, t, acc);
    }
    A[e] = scale * exp(acc) + (a == b ? diag_add : 0.0);
}

// ------------------------------------------------- derivative products dK.W
// FP32 entries (direct differences, exp2), FP32 accumulation inside a column
// range, FP64 across ranges.  With x' = (x - mu)/l * sqrt(log2(e)/2):
//   (x_ir - x_jr)^2 / l_r^2 = 2/log2(e) * t_r^2,  t_r = x'_ir - x'_jr.
// Output slots: ARD: r = 0..d-1 then log s^2 (slot d); isotropic: slot 0 is
// the sum over r, slot 1 is log s^2.
template <int DP, int CB>
__global__ void __launch_bounds__(KT)
    dkv_kernel(const float* __restrict__ xs, int64_t n, int nq, int ard, float c0,
               const float* __restrict__ W, int64_t ldw, int ncols, float* __restrict__ part,
               int64_t ldp, int64_t cps) {
    __shared__ __align__(16) float sx[TJ * DP];
    __shared__ __align__(16) float sw[TJ * CB];
    const int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * cps;
    const int64_t j1 = min(n, j0 + cps);
    constexpr float kScale = 1.3862943611198906f;  // 2 / log2(e) = 2 ln 2
    float xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < n) ? xs[i * DP + q] : 0.f;
    float acc[DP + 1][CB];
#pragma unroll
    for (int q = 0; q <= DP; ++q)
#pragma unroll
        for (int k = 0; k < CB; ++k) acc[q][k] = 0.f;
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        const int jn = (int)min((int64_t)TJ, j1 - jt);
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DP; e += KT) {
            const int jj = e / DP;
            sx[e] = (jj < jn) ? xs[(jt + jj) * DP + (e - jj * DP)] : 0.f;
        }
        for (int e = threadIdx.x; e < TJ * CB; e += KT) {
            const int k = e / TJ, jj = e - k * TJ;
            sw[jj * CB + k] = (jj < jn && k < ncols) ? W[(jt + jj) + (int64_t)k * ldw] : 0.f;
        }
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            float t2[DP];
            float a = c0;
#pragma unroll
            for (int q = 0; q < DP; ++q) {
                const float t = xi[q] - sx[jj * DP + q];
                t2[q] = t * t;
                a -= t2[q];
            }
            const float e = kexp<float>(a);
            float ew[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                ew[k] = e * sw[jj * CB + k];
                acc[DP][k] += ew[k];
            }
#pragma unroll
            for (int q = 0; q < DP; ++q)
#pragma unroll
                for (int k = 0; k < CB; ++k) acc[q][k] = fmaf(t2[q], ew[k], acc[q][k]);
        }
    }
    if (i >= n) return;
    for (int k = 0; k < ncols; ++k) {
        float* base = part + ((int64_t)blockIdx.y * CB + k) * (int64_t)(nq)*ldp;
        if (ard) {
#pragma unroll
            for (int q = 0; q < DP; ++q)
                if (q < nq - 1) base[(int64_t)q * ldp + i] = kScale * acc[q][k];
        } else {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < DP; ++q) s += acc[q][k];
            base[i] = kScale * s;
        }
        base[(int64_t)(nq - 1) * ldp + i] = acc[DP][k];
    }
}

__global__ void dkv_reduce_kernel(const float* __restrict__ part, int64_t ldp, int nsplit, int cb,
                                  int nq, int ncols, double* __restrict__ G, int64_t ldg,
                                  int64_t c_total, int k0, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y, k = blockIdx.z;
    if (i >= n || k >= ncols) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp)
        s += (double)part[(((int64_t)sp * cb + k) * nq + q) * ldp + i];
    G[(int64_t)q * ldg * c_total + (int64_t)(k0 + k) * ldg + i] = s;
}

template <int DP>
void dkv_launch(int cb, const float* xs, int64_t n, int nq, int ard, float c0, const float* W,
                int64_t ldw, int ncols, float* part, const Split& s, cudaStream_t st) {
    dim3 grid(s.nrb, s.nsplit);
    switch (cb) {
        case 1:
            dkv_kernel<DP, 1><<<grid, KT, 0, st>>>(xs, n, nq, ard, c0, W, ldw, ncols, part, s.ldp,
                                                   s.cps);
            break;
        case 2:
            dkv_kernel<DP, 2><<<grid, KT, 0, st>>>(xs, n, nq, ard, c0, W, ldw, ncols, part, s.ldp,
                                                   s.cps);
            break;
        case 4:
            dkv_kernel<DP, 4><<<grid, KT, 0, st>>>(xs, n, nq, ard, c0, W, ldw, ncols, part, s.ldp,
                                                   s.cps);
            break;
        default: fail(KPCG_ERR_ARG, "internal: bad dkv column block");
    }
    KPCG_LAUNCHED("dkv_kernel");
}

// The derivative products in native FP64 (inputs x' scaled by sqrt(1/2), so
// K_ij = exp(c0 - sum_r t_r^2), t = x'_i - x'_j, and (x_ir - x_jr)^2 / l_r^2 =
// 2 t_r^2).  The gradient's trace term w^T (dK r) sums products of a large,
// rough w = K_y^{-1} r with dK r and cancels most of their magnitude, so dK W
// needs FP64-class entries; FP32 entries leave errors of ~1e-3 relative on
// the smaller gradient entries.
template <int DP, int CB>
__global__ void __launch_bounds__(KT)
    dkv64_kernel(const double* __restrict__ xs, int64_t n, int nq, int ard, double c0,
                 const double* __restrict__ W, int64_t ldw, int ncols, double* __restrict__ part,
                 int64_t ldp, int64_t cps) {
    __shared__ double sx[TJ * DP];
    __shared__ double sw[TJ * CB];
    const int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * cps;
    const int64_t j1 = min(n, j0 + cps);
    double xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < n) ? xs[i * DP + q] : 0.0;
    double acc[DP + 1][CB];
#pragma unroll
    for (int q = 0; q <= DP; ++q)
#pragma unroll
        for (int k = 0; k < CB; ++k) acc[q][k] = 0.0;
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        const int jn = (int)min((int64_t)TJ, j1 - jt);
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DP; e += KT) {
            const int jj = e / DP;
            sx[e] = (jj < jn) ? xs[(jt + jj) * DP + (e - jj * DP)] : 0.0;
        }
        for (int e = threadIdx.x; e < TJ * CB; e += KT) {
            const int k = e / TJ, jj = e - k * TJ;
            sw[jj * CB + k] = (jj < jn && k < ncols) ? W[(jt + jj) + (int64_t)k * ldw] : 0.0;
        }
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            double t2[DP];
            double a = c0;
#pragma unroll
            for (int q = 0; q < DP; ++q) {
                const double t = xi[q] - sx[jj * DP + q];
                t2[q] = t * t;
                a -= t2[q];
            }
            const double e = exp(a);
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const double ew = e * sw[jj * CB + k];
                acc[DP][k] += ew;
#pragma unroll
                for (int q = 0; q < DP; ++q) acc[q][k] = fma(t2[q], ew, acc[q][k]);
            }
        }
    }
    if (i >= n) return;
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        if (k >= ncols) break;
        double* base = part + ((int64_t)blockIdx.y * CB + k) * (int64_t)(nq)*ldp;
        if (ard) {
#pragma unroll
            for (int q = 0; q < DP; ++q)
                if (q < nq - 1) base[(int64_t)q * ldp + i] = 2.0 * acc[q][k];
        } else {
            double sum = 0.0;
#pragma unroll
            for (int q = 0; q < DP; ++q) sum += acc[q][k];
            base[i] = 2.0 * sum;
        }
        base[(int64_t)(nq - 1) * ldp + i] = acc[DP][k];
    }
}

__global__ void dkv64_reduce_kernel(const double* __restrict__ part, int64_t ldp, int nsplit,
                                    int cb, int nq, int ncols, double* __restrict__ G,
                                    int64_t ldg, int64_t c_total, int k0, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y, k = blockIdx.z;
    if (i >= n || k >= ncols) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[(((int64_t)sp * cb + k) * nq + q) * ldp + i];
    G[(int64_t)q * ldg * c_total + (int64_t)(k0 + k) * ldg + i] = s;
}

template <int DP>
void dkv64_launch(int cb, const double* xs, int64_t n, int nq, int ard, double c0,
                  const double* W, int64_t ldw, int ncols, double* part, const Split& s,
                  cudaStream_t st) {
    dim3 grid(s.nrb, s.nsplit);
    if (cb == 1)
        dkv64_kernel<DP, 1><<<grid, KT, 0, st>>>(xs, n, nq, ard, c0, W, ldw, ncols, part, s.ldp,
                                                 s.cps);
    else
        dkv64_kernel<DP, 2><<<grid, KT, 0, st>>>(xs, n, nq, ard, c0, W, ldw, ncols, part, s.ldp,
                                                 s.cps);
    KPCG_LAUNCHED("dkv64_kernel");
}

}  // namespace

void dkv_f64(const double* xs, int64_t n, int dp, int d, int ard, double c0, const double* W,
             int64_t ldw, int c, double* G, int64_t ldg, KvWorkspace& ws, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    const int nq = (ard ? d : 1) + 1;
    const Split s = plan(n, KT);
    const int max_cb = 2;
    double* part = ws.part64.need((size_t)s.nsplit * max_cb * nq * s.ldp);
    for (int k0 = 0; k0 < c;) {
        const int cb = (c - k0) >= 2 ? 2 : 1;
        const double* Wk = W + (int64_t)k0 * ldw;
        switch (dp) {
            case 4: dkv64_launch<4>(cb, xs, n, nq, ard, c0, Wk, ldw, cb, part, s, st); break;
            case 8: dkv64_launch<8>(cb, xs, n, nq, ard, c0, Wk, ldw, cb, part, s, st); break;
            case 12: dkv64_launch<12>(cb, xs, n, nq, ard, c0, Wk, ldw, cb, part, s, st); break;
            case 16: dkv64_launch<16>(cb, xs, n, nq, ard, c0, Wk, ldw, cb, part, s, st); break;
            case 32: dkv64_launch<32>(cb, xs, n, nq, ard, c0, Wk, ldw, cb, part, s, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        dim3 rg((unsigned)((n + 255) / 256), (unsigned)nq, (unsigned)cb);
        dkv64_reduce_kernel<<<rg, 256, 0, st>>>(part, s.ldp, s.nsplit, cb, nq, cb, G, ldg, c, k0,
                                                n);
        KPCG_LAUNCHED("dkv64_reduce_kernel");
        k0 += cb;
    }
}

namespace {
}  // namespace

size_t kv_f64_scratch_elems(int64_t n) {
    if (n <= 0) return 0;
    const Split s = plan(n, KT);
    return (size_t)s.nsplit * 4 * (size_t)s.ldp;
}

void kv_f64_into(const double* xs, int64_t n, int dp, double c0, double noise, const double* V,
                 int64_t ldv, int c, double* O, int64_t ldo, double* part, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    const Split s = plan(n, KT);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        const double* Vk = V + (int64_t)k0 * ldv;
        switch (dp) {
            case 4: launch_cb<double, 4>(cb, xs, n, c0, Vk, ldv, ncols, part, s, 1, st); break;
            case 8: launch_cb<double, 8>(cb, xs, n, c0, Vk, ldv, ncols, part, s, 1, st); break;
            case 12: launch_cb<double, 12>(cb, xs, n, c0, Vk, ldv, ncols, part, s, 1, st); break;
            case 16: launch_cb<double, 16>(cb, xs, n, c0, Vk, ldv, ncols, part, s, 1, st); break;
            case 32: launch_cb<double, 32>(cb, xs, n, c0, Vk, ldv, ncols, part, s, 1, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        dim3 rg((unsigned)((n + 255) / 256), (unsigned)ncols);
        kv_reduce_kernel<double><<<rg, 256, 0, st>>>(part, s.ldp, s.nsplit, cb, ncols, Vk, ldv,
                                                     noise, nullptr, 0, O + (int64_t)k0 * ldo,
                                                     ldo, n);
        KPCG_LAUNCHED("kv_reduce_kernel");
        k0 += ncols;
    }
}

void kv_f64(const double* xs, int64_t n, int dp, double c0, double noise, const double* V,
            int64_t ldv, int c, const double* B, int64_t ldb, double* O, int64_t ldo,
            KvWorkspace& ws, cudaStream_t st) {
    kv_generic<double>(xs, n, dp, c0, noise, V, ldv, c, B, ldb, O, ldo, ws.part64, st);
}

void kv_f32(const float* xs, int64_t n, int dp, float c0, float noise, const float* V,
            int64_t ldv, int c, float* O, int64_t ldo, KvWorkspace& ws, cudaStream_t st) {
    kv_generic<float>(xs, n, dp, c0, noise, V, ldv, c, nullptr, 0, O, ldo, ws.part32, st);
}

void kxu_f32(const float* xs, int64_t n, const float* us, int64_t m, int dp, float c0,
             float* KXU, cudaStream_t st) {
    const int64_t tot = n * m;
    if (tot == 0) return;
    kxu_f32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(xs, n, us, m, dp, c0, KXU);
    KPCG_LAUNCHED("kxu_f32_kernel");
}

void kxu_pair_f64(const double* xs, int64_t n, const double* us, int64_t m, int dp, double c0,
                  float2* KXU, cudaStream_t st) {
    const int64_t tot = n * m;
    if (tot == 0) return;
    kxu_pair_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(xs, n, us, m, dp, c0, KXU);
    KPCG_LAUNCHED("kxu_pair_kernel");
}

void kuu_f64(const double* us, int64_t m, int dp, double c0, double scale, double diag_add,
             double* A, cudaStream_t st) {
    const int64_t tot = m * m;
    if (tot == 0) return;
    kuu_f64_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(us, m, dp, c0, scale, diag_add,
                                                                  A);
    KPCG_LAUNCHED("kuu_f64_kernel");
}

void dkv_f32(const float* xs, int64_t n, int dp, int d, int ard, float c0, const float* W,
             int64_t ldw, int c, double* G, int64_t ldg, KvWorkspace& ws, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    const int nq = (ard ? d : 1) + 1;
    const Split s = plan(n, KT);
    const int max_cb = 4;
    float* part = ws.part32.need((size_t)s.nsplit * max_cb * nq * s.ldp);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        const float* Wk = W + (int64_t)k0 * ldw;
        switch (dp) {
            case 4: dkv_launch<4>(cb, xs, n, nq, ard, c0, Wk, ldw, ncols, part, s, st); break;
            case 8: dkv_launch<8>(cb, xs, n, nq, ard, c0, Wk, ldw, ncols, part, s, st); break;
            case 12: dkv_launch<12>(cb, xs, n, nq, ard, c0, Wk, ldw, ncols, part, s, st); break;
            case 16: dkv_launch<16>(cb, xs, n, nq, ard, c0, Wk, ldw, ncols, part, s, st); break;
            case 32: dkv_launch<32>(cb, xs, n, nq, ard, c0, Wk, ldw, ncols, part, s, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        dim3 rg((unsigned)((n + 255) / 256), (unsigned)nq, (unsigned)ncols);
        dkv_reduce_kernel<<<rg, 256, 0, st>>>(part, s.ldp, s.nsplit, cb, nq, ncols, G, ldg, c, k0,
                                              n);
        KPCG_LAUNCHED("dkv_reduce_kernel");
        k0 += ncols;
    }
}

}  // namespace kpcg
