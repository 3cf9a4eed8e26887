// kpcg_matvec_f64_noalloc: the native-FP64 kernel product without any device
// allocation.  Its scratch -- column means, the scaled inputs and the split
// partial sums -- lives in one file-scope __device__ array of fixed size that
// every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "kpcg_internal.cuh"

namespace kpcg {
namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_mu;
void* g_ptr[kMaxDev] = {};

struct InvEll {
    double v[32];
};

__global__ void na_colmean_kernel(const float* __restrict__ X, int64_t n, int d,
                                  double* __restrict__ mu) {
    __shared__ double sh[256];
    const int q = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)X[i * d + q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mu[q] = sh[0] / (double)n;
}

__global__ void na_prescale_kernel(const float* __restrict__ X, int64_t n, int d, int dp,
                                   const double* __restrict__ mu, InvEll inv, double g,
                                   double* __restrict__ xs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * dp) return;
    const int64_t i = e / dp;
    const int q = (int)(e - i * dp);
    double v = 0.0;
    if (q < d) v = ((double)X[i * d + q] - mu[q]) * inv.v[q];
    xs[e] = v * g;
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
unsigned char* scratch_for_current_device() {
    int dev = 0;
    KPCG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) fail(KPCG_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        KPCG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        if (!p) fail(KPCG_ERR_CUDA, "cudaGetSymbolAddress returned a null address");
        g_ptr[dev] = p;
    }
    return static_cast<unsigned char*>(g_ptr[dev]);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace kpcg

extern "C" kpcg_status kpcg_matvec_f64_noalloc(const float* X, int64_t n, int32_t d,
                                               const double* log_theta, int32_t ard,
                                               double noise_var, const double* V, int64_t ldv,
                                               int32_t c, double* O, int64_t ldo, void* stream) {
    using namespace kpcg;
    try {
        if (!X || !log_theta || !V || !O) fail(KPCG_ERR_ARG, "NULL argument");
        if (n < 1 || c < 0 || ldv < n || ldo < n) fail(KPCG_ERR_ARG, "bad sizes");
        // n is capped before any size arithmetic, so the scratch plan below
        // cannot wrap around
        if (n > ((int64_t)1 << 31)) fail(KPCG_ERR_ARG, "n too large");
        check_dev_ptr(X, "X");
        check_dev_ptr(V, "V");
        check_dev_ptr(O, "O");
        if ((reinterpret_cast<uintptr_t>(X) & 3u) != 0)
            fail(KPCG_ERR_ARG, "X must be 4-byte aligned");
        if ((reinterpret_cast<uintptr_t>(V) & 7u) != 0 || (reinterpret_cast<uintptr_t>(O) & 7u) != 0)
            fail(KPCG_ERR_ARG, "V and O must be 8-byte aligned");
        const int dp = padded_dim(d);
        if (d < 1 || dp < 0) fail(KPCG_ERR_ARG, "d must be in [1, 32]");
        if (!(noise_var > 0.0) || !std::isfinite(noise_var))
            fail(KPCG_ERR_ARG, "noise_var must be > 0");
        const int nt = ard ? d + 1 : 2;
        for (int i = 0; i < nt; ++i)
            if (!std::isfinite(log_theta[i])) fail(KPCG_ERR_ARG, "log_theta has a non-finite entry");
        if (c == 0) return KPCG_OK;
        // scratch plan: [mu (32 doubles)] [x' n x dp] [partial sums]
        const size_t b_mu = align256(32 * sizeof(double));
        const size_t b_xs = align256((size_t)n * dp * sizeof(double));
        const size_t b_part = align256(kv_f64_scratch_elems(n) * sizeof(double));
        if (b_mu + b_xs + b_part > kScratchBytes)
            fail(KPCG_ERR_ARG, "n = " + std::to_string(n) + ", d = " + std::to_string(d) +
                                   " needs " + std::to_string(b_mu + b_xs + b_part) +
                                   " bytes of scratch; the static scratch holds " +
                                   std::to_string(kScratchBytes));
        unsigned char* base = scratch_for_current_device();
        double* mu = reinterpret_cast<double*>(base);
        double* xs = reinterpret_cast<double*>(base + b_mu);
        double* part = reinterpret_cast<double*>(base + b_mu + b_xs);
        cudaStream_t st = (cudaStream_t)stream;
        InvEll inv{};
        for (int q = 0; q < d; ++q) inv.v[q] = std::exp(-(ard ? log_theta[q] : log_theta[0]));
        const double s2 = std::exp(log_theta[nt - 1]);
        na_colmean_kernel<<<d, 256, 0, st>>>(X, n, d, mu);
        KPCG_LAUNCHED("na_colmean_kernel");
        na_prescale_kernel<<<(unsigned)((n * dp + 255) / 256), 256, 0, st>>>(X, n, d, dp, mu, inv,
                                                                            std::sqrt(0.5), xs);
        KPCG_LAUNCHED("na_prescale_kernel");
        kv_f64_into(xs, n, dp, std::log(s2), noise_var, V, ldv, c, O, ldo, part, st);
        KPCG_CUDA(cudaStreamSynchronize(st));
        return KPCG_OK;
    } catch (const Error& e) {
        set_handleless_error(e.msg);
        return e.status;
    }
}
