// Vector steps and scalars of batched preconditioned CG (Algorithm 1).
//
// Each of the c columns of a block runs its own CG: its own alpha, beta and
// rho, its own stop test, and it is frozen (alpha = beta = 0) once it stops.
// Dot products accumulate in FP64 whatever the vector type: products are
// formed in FP64 and reduced per CTA, the per-CTA partials are then added
// in a fixed order by one small kernel that also runs the scalar logic
// (deterministic, no atomics).  Scalars never leave the device; the host
// only polls the count of active columns.
#include <cuda_runtime.h>

#include "kpcg_internal.cuh"

namespace kpcg {
namespace {

constexpr int DT = 256;  // threads of the reduction kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

template <typename T>
__global__ void __launch_bounds__(DT)
    dot_kernel(const T* __restrict__ A, int64_t lda, const T* __restrict__ B, int64_t ldb,
               int64_t n, double* __restrict__ partial, int nblk) {
    __shared__ double sh[DT / 32];
    const int k = blockIdx.y;
    const T* a = A + (int64_t)k * lda;
    const T* b = B + (int64_t)k * ldb;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x; i < n; i += (int64_t)nblk * DT)
        s = fma((double)a[i], (double)b[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(int64_t)k * nblk + blockIdx.x] = s;
}

// x += alpha p; r -= alpha q; partial ||r||^2.
template <typename T>
__global__ void __launch_bounds__(DT)
    update_xr_kernel(T* __restrict__ x, int64_t ldx, T* __restrict__ r, int64_t ldr,
                     const T* __restrict__ p, int64_t ldp, const T* __restrict__ q, int64_t ldq,
                     int64_t n, const double* __restrict__ alpha, double* __restrict__ partial,
                     int nblk) {
    __shared__ double sh[DT / 32];
    const int k = blockIdx.y;
    const double al = alpha[k];
    const T a = (T)al;
    T* xk = x + (int64_t)k * ldx;
    T* rk = r + (int64_t)k * ldr;
    const T* pk = p + (int64_t)k * ldp;
    const T* qk = q + (int64_t)k * ldq;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DT + threadIdx.x; i < n; i += (int64_t)nblk * DT) {
        T ri = rk[i];
        if (al != 0.0) {
            xk[i] = fma(a, pk[i], xk[i]);
            ri = fma(-a, qk[i], ri);
            rk[i] = ri;
        }
        s = fma((double)ri, (double)ri, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(int64_t)k * nblk + blockIdx.x] = s;
}

template <typename T>
__global__ void update_p_kernel(T* __restrict__ p, int64_t ldp, const T* __restrict__ z,
                                int64_t ldz, int64_t n, const double* __restrict__ beta,
                                const int* __restrict__ active) {
    const int k = blockIdx.y;
    if (!active[k]) return;
    const T b = (T)beta[k];
    T* pk = p + (int64_t)k * ldp;
    const T* zk = z + (int64_t)k * ldz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        pk[i] = fma(b, pk[i], zk[i]);
}

// One thread per column: fixed-order sum of the partials, then the scalar
// step of Algorithm 1 selected by mode.
__global__ void finalize_kernel(const double* __restrict__ partial, int nblk, int c, int mode,
                                CgScalars s, double tol, int tol_mode, int64_t n,
                                int* __restrict__ host_flags) {
    __shared__ int n_active, n_broken;
    if (threadIdx.x == 0) {
        n_active = 0;
        n_broken = 0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < c; k += blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < nblk; ++b) v += partial[(int64_t)k * nblk + b];
        switch (mode) {
            case FIN_NORM_B:  // v = ||b||^2: threshold and activity
                s.bnorm2[k] = v;
                s.thr2[k] = (tol_mode == 1) ? (double)n * tol : tol * tol * v;
                s.iters[k] = 0;
                s.active[k] = (v > 0.0) ? 1 : 0;
                break;
            case FIN_RHO0:  // v = r0^T z0
                s.rho[k] = v;
                break;
            case FIN_ALPHA:  // v = p^T K_y p
                if (s.active[k]) {
                    if (!(v > 0.0) || !isfinite(v) || !isfinite(s.rho[k])) {
                        s.alpha[k] = 0.0;
                        s.active[k] = 0;
                        s.iters[k] = -1 - s.iters[k];  // breakdown marker
                        atomicAdd(&n_broken, 1);
                    } else {
                        s.alpha[k] = s.rho[k] / v;
                    }
                } else {
                    s.alpha[k] = 0.0;
                }
                break;
            case FIN_RR:  // v = ||r||^2 after the update
                s.rr[k] = v;
                if (s.active[k]) {
                    s.iters[k] += 1;
                    if (v <= s.thr2[k]) s.active[k] = 0;
                }
                break;
            case FIN_BETA:  // v = r^T z
                if (s.active[k]) {
                    s.beta[k] = v / s.rho[k];
                    s.rho[k] = v;
                } else {
                    s.beta[k] = 0.0;
                }
                break;
        }
        if (s.active[k]) atomicAdd(&n_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s.flags[0] = n_active;
        if (mode == FIN_ALPHA) s.flags[1] += n_broken;
        if (host_flags) {
            host_flags[0] = n_active;
            host_flags[1] = s.flags[1];
        }
    }
}

template <typename T>
__global__ void copy_cols_kernel(T* __restrict__ dst, int64_t ldd, const T* __restrict__ src,
                                 int64_t lds, int64_t n) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i + (int64_t)k * ldd] = src[i + (int64_t)k * lds];
}

// dst = src * s_k (invert = 0) or src / s_k (invert = 1), with type change.
template <typename TD, typename TS>
__global__ void convert_scale_kernel(TD* __restrict__ dst, int64_t ldd, const TS* __restrict__ src,
                                     int64_t lds, int64_t n, const double* __restrict__ colscale,
                                     int invert) {
    const int k = blockIdx.y;
    double f = colscale ? colscale[k] : 1.0;
    if (colscale && invert) f = (f > 0.0) ? 1.0 / f : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i + (int64_t)k * ldd] = (TD)((double)src[i + (int64_t)k * lds] * f);
}

__global__ void axpy_scaled_kernel(double* __restrict__ X, int64_t ldx, const float* __restrict__ D,
                                   int64_t ldd, int64_t n, const double* __restrict__ colscale) {
    const int k = blockIdx.y;
    const double f = colscale[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        X[i + (int64_t)k * ldx] += f * (double)D[i + (int64_t)k * ldd];
}

__global__ void axpy_cols_kernel(double* __restrict__ Y, int64_t ldy, const double* __restrict__ X,
                                 int64_t ldx, int64_t n, const double* __restrict__ coef) {
    const int k = blockIdx.y;
    const double f = coef[k];
    if (f == 0.0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        Y[i + (int64_t)k * ldy] = fma(f, X[i + (int64_t)k * ldx], Y[i + (int64_t)k * ldy]);
}

unsigned grid_x(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int dot_blocks(int64_t n) {
    int64_t b = (n + DT * 8 - 1) / (DT * 8);
    if (b > 296) b = 296;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
void dot_cols(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t n, int c,
              double* partial, int nblk, cudaStream_t st) {
    dot_kernel<T><<<dim3(nblk, c), DT, 0, st>>>(A, lda, B, ldb, n, partial, nblk);
    KPCG_LAUNCHED("dot_kernel");
}

void finalize(const double* partial, int nblk, int c, int mode, CgScalars s, double tol,
              int tol_mode, int64_t n, int* host_flags, cudaStream_t st) {
    finalize_kernel<<<1, 256, 0, st>>>(partial, nblk, c, mode, s, tol, tol_mode, n, host_flags);
    KPCG_LAUNCHED("finalize_kernel");
}

template <typename T>
void update_xr(T* x, int64_t ldx, T* r, int64_t ldr, const T* p, int64_t ldp, const T* q,
               int64_t ldq, int64_t n, int c, const double* alpha, double* partial, int nblk,
               cudaStream_t st) {
    update_xr_kernel<T><<<dim3(nblk, c), DT, 0, st>>>(x, ldx, r, ldr, p, ldp, q, ldq, n, alpha,
                                                      partial, nblk);
    KPCG_LAUNCHED("update_xr_kernel");
}

template <typename T>
void update_p(T* p, int64_t ldp, const T* z, int64_t ldz, int64_t n, int c, const double* beta,
              const int* active, cudaStream_t st) {
    update_p_kernel<T><<<dim3(grid_x(n), c), 256, 0, st>>>(p, ldp, z, ldz, n, beta, active);
    KPCG_LAUNCHED("update_p_kernel");
}

template <typename T>
void copy_cols(T* dst, int64_t ldd, const T* src, int64_t lds, int64_t n, int c, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    copy_cols_kernel<T><<<dim3(grid_x(n), c), 256, 0, st>>>(dst, ldd, src, lds, n);
    KPCG_LAUNCHED("copy_cols_kernel");
}

template <typename TD, typename TS>
void convert_scale_cols(TD* dst, int64_t ldd, const TS* src, int64_t lds, int64_t n, int c,
                        const double* colscale, int invert, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    convert_scale_kernel<TD, TS><<<dim3(grid_x(n), c), 256, 0, st>>>(dst, ldd, src, lds, n,
                                                                    colscale, invert);
    KPCG_LAUNCHED("convert_scale_kernel");
}

void axpy_scaled_f64(double* X, int64_t ldx, const float* D, int64_t ldd, int64_t n, int c,
                     const double* colscale, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    axpy_scaled_kernel<<<dim3(grid_x(n), c), 256, 0, st>>>(X, ldx, D, ldd, n, colscale);
    KPCG_LAUNCHED("axpy_scaled_kernel");
}

void axpy_cols_f64(double* Y, int64_t ldy, const double* X, int64_t ldx, int64_t n, int c,
                   const double* coef, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    axpy_cols_kernel<<<dim3(grid_x(n), c), 256, 0, st>>>(Y, ldy, X, ldx, n, coef);
    KPCG_LAUNCHED("axpy_cols_kernel");
}

void fill_zero_cols(void* p, size_t elem, int64_t ld, int64_t n, int c, cudaStream_t st) {
    if (n <= 0 || c <= 0) return;
    KPCG_CUDA(cudaMemset2DAsync(p, (size_t)ld * elem, 0, (size_t)n * elem, (size_t)c, st));
}

template void dot_cols<float>(const float*, int64_t, const float*, int64_t, int64_t, int, double*,
                              int, cudaStream_t);
template void dot_cols<double>(const double*, int64_t, const double*, int64_t, int64_t, int,
                               double*, int, cudaStream_t);
template void update_xr<float>(float*, int64_t, float*, int64_t, const float*, int64_t,
                               const float*, int64_t, int64_t, int, const double*, double*, int,
                               cudaStream_t);
template void update_xr<double>(double*, int64_t, double*, int64_t, const double*, int64_t,
                                const double*, int64_t, int64_t, int, const double*, double*, int,
                                cudaStream_t);
template void update_p<float>(float*, int64_t, const float*, int64_t, int64_t, int,
                              const double*, const int*, cudaStream_t);
template void update_p<double>(double*, int64_t, const double*, int64_t, int64_t, int,
                               const double*, const int*, cudaStream_t);
template void copy_cols<float>(float*, int64_t, const float*, int64_t, int64_t, int, cudaStream_t);
template void copy_cols<double>(double*, int64_t, const double*, int64_t, int64_t, int,
                                cudaStream_t);
template void convert_scale_cols<float, double>(float*, int64_t, const double*, int64_t, int64_t,
                                                int, const double*, int, cudaStream_t);
template void convert_scale_cols<double, float>(double*, int64_t, const float*, int64_t, int64_t,
                                                int, const double*, int, cudaStream_t);
template void convert_scale_cols<double, double>(double*, int64_t, const double*, int64_t,
                                                 int64_t, int, const double*, int, cudaStream_t);

}  // namespace kpcg
