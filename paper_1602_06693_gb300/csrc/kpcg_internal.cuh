// Internal declarations shared by the CUDA translation units of libkpcg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kpcg.h"

namespace kpcg {

// Thrown inside the library, converted to a status at the C boundary.
struct Error {
    kpcg_status status;
    std::string msg;
};

[[noreturn]] void fail(kpcg_status s, const std::string& msg);
void set_handleless_error(const std::string& msg);
void cuda_check(cudaError_t e, const char* what, const char* file, int line);
#define KPCG_CUDA(call) ::kpcg::cuda_check((call), #call, __FILE__, __LINE__)
// Checks a kernel launch and counts it (per host thread).
void note_launch();
// count k kernel launches made by replaying a captured graph
void note_launches(long long k);
long long launch_count();
// KPCG_TRACE=1 in the environment: the solvers print one line per outer step
// (worst relative residual, iterations so far) to stderr.
bool trace_on();
// KPCG_ERR_ARG unless p is a non-NULL device (or managed) pointer.
void check_dev_ptr(const void* p, const char* name);
#define KPCG_LAUNCHED(name) \
    (::kpcg::note_launch(), ::kpcg::cuda_check(cudaGetLastError(), name, __FILE__, __LINE__))

// A device allocation owned by RAII.
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t count = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        count = 0;
    }
    // Grow to at least n elements (contents are not preserved).
    T* need(size_t n) {
        if (n <= count && p) return p;
        release();
        size_t bytes = (n ? n : 1) * sizeof(T);
        cudaError_t e = cudaMalloc((void**)&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            fail(KPCG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
        count = n;
        return p;
    }
};

// Padded feature dimension used by the kernels: 4, 8, 12, 16 or 32.
int padded_dim(int d);

// ---------------------------------------------------------------- K.V (kv.cu)
// Scaled inputs: the kernels see x' = (x - mu) / l * g with g = sqrt(1/2) for
// FP64 (entries exp(c0 - |x'_i - x'_j|^2), c0 = log s^2) and
// g = sqrt(log2(e)/2) for FP32 (entries exp2(c0 - |x'_i - x'_j|^2),
// c0 = log2 s^2).  Rows are padded with zeros to dp columns.
struct KvWorkspace {
    DevBuf<float> part32;
    DevBuf<double> part64;
};

// O = K V + noise V  (or, when B != nullptr, O = B - (K V + noise V)).
void kv_f64(const double* xs, int64_t n, int dp, double c0, double noise, const double* V,
            int64_t ldv, int c, const double* B, int64_t ldb, double* O, int64_t ldo,
            KvWorkspace& ws, cudaStream_t st);
// The FP64 product with caller-provided partial-sum scratch of at least
// kv_f64_scratch_elems(n) doubles (column blocks of up to four).
size_t kv_f64_scratch_elems(int64_t n);
void kv_f64_into(const double* xs, int64_t n, int dp, double c0, double noise, const double* V,
                 int64_t ldv, int c, double* O, int64_t ldo, double* part, cudaStream_t st);
void kv_f32(const float* xs, int64_t n, int dp, float c0, float noise, const float* V,
            int64_t ldv, int c, float* O, int64_t ldo, KvWorkspace& ws, cudaStream_t st);

// Tensor-core variant (kv_tc.cu).  kv_tc_supported reports whether the
// input dimension fits the augmented K-dimension (6d + 6 <= 128, i.e.
// d <= 20); there is no fallback.
bool kv_tc_supported(int d);

// Cross-kernel block K(X, U) (n x m row-major), FP32 entries from FP32-scaled inputs.
void kxu_f32(const float* xs, int64_t n, const float* us, int64_t m, int dp, float c0,
             float* KXU, cudaStream_t st);
// Cross block K(X, U) (n x m row-major) with FP64 entries stored as FP32 pairs.
void kxu_pair_f64(const double* xs, int64_t n, const double* us, int64_t m, int dp, double c0,
                  float2* KXU, cudaStream_t st);
// Square FP64 block s2 * K(U, U) (m x m row-major) plus diag_add on the diagonal.
void kuu_f64(const double* us, int64_t m, int dp, double c0, double scale, double diag_add,
             double* A, cudaStream_t st);

// dK/dtheta . W products: n_theta blocks of n x c (FP64 out, leading dim ldg,
// block q at G + q*ldg*c): per dimension r (ARD) or pooled (isotropic), then
// log s^2.  FP32 entries and FP32 accumulation within a column range.
void dkv_f32(const float* xs, int64_t n, int dp, int d, int ard, float c0, const float* W,
             int64_t ldw, int c, double* G, int64_t ldg, KvWorkspace& ws, cudaStream_t st);
// The same products with FP64 entries and sums (W in FP64): what the gradient
// uses, since its trace term cancels most of the magnitude of dK W.
void dkv_f64(const double* xs, int64_t n, int dp, int d, int ard, double c0, const double* W,
             int64_t ldw, int c, double* G, int64_t ldg, KvWorkspace& ws, cudaStream_t st);

// --------------------------------------------------------------- CG (cg.cu)
// Per-column scalars of the batched PCG, device resident.
struct CgScalars {
    double* rho;     // r^T z
    double* alpha;   // step
    double* beta;
    double* rr;      // ||r||^2
    double* thr2;    // stop threshold on ||r||^2
    double* bnorm2;  // ||b||^2
    int* active;     // 1 while the column iterates
    int* iters;      // iterations done by the column
    int* flags;      // [0] active count, [1] breakdown count
};

enum FinalizeMode { FIN_NORM_B = 0, FIN_RHO0 = 1, FIN_ALPHA = 2, FIN_RR = 3, FIN_BETA = 4 };

template <typename T>
void dot_cols(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t n, int c,
              double* partial, int nblk, cudaStream_t st);
// Reduce partial dots and run the per-column scalar logic of Algorithm 1.
void finalize(const double* partial, int nblk, int c, int mode, CgScalars s, double tol,
              int tol_mode, int64_t n, int* host_flags, cudaStream_t st);
template <typename T>
void update_xr(T* x, int64_t ldx, T* r, int64_t ldr, const T* p, int64_t ldp, const T* q,
               int64_t ldq, int64_t n, int c, const double* alpha, double* partial, int nblk,
               cudaStream_t st);
template <typename T>
void update_p(T* p, int64_t ldp, const T* z, int64_t ldz, int64_t n, int c, const double* beta,
              const int* active, cudaStream_t st);
template <typename T>
void copy_cols(T* dst, int64_t ldd, const T* src, int64_t lds, int64_t n, int c, cudaStream_t st);
template <typename TD, typename TS>
void convert_scale_cols(TD* dst, int64_t ldd, const TS* src, int64_t lds, int64_t n, int c,
                        const double* colscale, int invert, cudaStream_t st);
void axpy_scaled_f64(double* X, int64_t ldx, const float* D, int64_t ldd, int64_t n, int c,
                     const double* colscale, cudaStream_t st);
// Y[:, k] += coef[k] X[:, k]  (device coefficients).
void axpy_cols_f64(double* Y, int64_t ldy, const double* X, int64_t ldx, int64_t n, int c,
                   const double* coef, cudaStream_t st);
void fill_zero_cols(void* p, size_t elem, int64_t ld, int64_t n, int c, cudaStream_t st);
int dot_blocks(int64_t n);

// ------------------------------------------------------ preconditioners
struct PrecondState;
void precond_apply_f64(const PrecondState& P, const double* R, int64_t ldr, int c, double* Z,
                       int64_t ldz, cudaStream_t st);
void precond_apply_f32(const PrecondState& P, const float* R, int64_t ldr, int c, float* Z,
                       int64_t ldz, cudaStream_t st);

}  // namespace kpcg
