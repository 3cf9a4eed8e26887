// kpcg_probe_rates: measured issue rates of the pipes the ALU-bound kernels
// use, for their rooflines.  The products of K with vectors (Sec. 2.1) are
// bound by FP32 arithmetic, the MUFU exp2 or FP64 arithmetic rather than by
// memory, and the vendor documents none of these rates for this part; this
// entry point measures them on the device it runs on.
//
// Each probe kernel runs 8 independent dependency chains per thread (enough
// to cover the pipe latency with 8 warps per scheduler) of a single
// instruction kind over a fixed number of rounds, on 8 CTAs of 256 threads
// per SM; the rate is lane-instructions divided by the CUDA-event time.  The
// first CTA also reads clock64() and %globaltimer at its start and end, which
// gives the SM clock under that load.  The chains feed a conditional store so
// that no instruction can be removed.
#include <cuda_runtime.h>

#include <cstdint>

#include "kpcg_internal.cuh"

namespace kpcg {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ __forceinline__ uint64_t probe_gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float probe_ex2(float a) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

// KIND 0: FP32 FMA, 1: MUFU ex2, 2: FP64 FMA.
template <int KIND>
__global__ void __launch_bounds__(kThreads) probe_kernel(int rounds, float seed, float* sink,
                                                         unsigned long long* clk) {
    unsigned long long c0 = 0, g0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        g0 = probe_gtimer();
    }
    if (KIND == 2) {
        double a[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = (double)seed + 1e-3 * (threadIdx.x + u);
        for (int r = 0; r < rounds; ++r)
#pragma unroll
            for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], 0.9999999, 1e-9);
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < kChains; ++u) s += a[u];
        if (s == 1234.5678) sink[threadIdx.x] = (float)s;
    } else {
        float a[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = seed + 1e-3f * (float)(threadIdx.x + u);
        for (int r = 0; r < rounds; ++r)
#pragma unroll
            for (int u = 0; u < kChains; ++u) {
                if (KIND == 0)
                    a[u] = fmaf(a[u], 0.9999999f, 1e-9f);
                else
                    a[u] = probe_ex2(-a[u]);  // converges to the fixed point of 2^-x
            }
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < kChains; ++u) s += a[u];
        if (s == 1234.5678f) sink[threadIdx.x] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64() - c0;
        clk[1] = probe_gtimer() - g0;
    }
}

template <int KIND>
double probe_one(int sms, cudaStream_t st, float* sink, unsigned long long* clk, double* mhz) {
    const int blocks = sms * 8;
    // calibrate to ~20 ms per timed launch
    int rounds = (KIND == 2) ? 256 : 4096;
    cudaEvent_t e0, e1;
    KPCG_CUDA(cudaEventCreate(&e0));
    KPCG_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int pass = 0; pass < 3; ++pass) {
        KPCG_CUDA(cudaEventRecord(e0, st));
        probe_kernel<KIND><<<blocks, kThreads, 0, st>>>(rounds, 0.5f, sink, clk);
        KPCG_LAUNCHED("probe_kernel");
        KPCG_CUDA(cudaEventRecord(e1, st));
        KPCG_CUDA(cudaEventSynchronize(e1));
        KPCG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (pass < 2 && ms < 20.f) {
            const double scale = 20.0 / (ms > 0.01f ? ms : 0.01f);
            const double want = rounds * (scale < 64.0 ? scale : 64.0);
            rounds = want > 1 << 26 ? 1 << 26 : (int)want;
        }
    }
    unsigned long long hc[2] = {0, 0};
    KPCG_CUDA(cudaMemcpyAsync(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    KPCG_CUDA(cudaEventDestroy(e0));
    KPCG_CUDA(cudaEventDestroy(e1));
    *mhz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;
    const double lanes = (double)blocks * kThreads * kChains * (double)rounds;
    return lanes / (ms * 1e-3);
}

}  // namespace
}  // namespace kpcg

extern "C" kpcg_status kpcg_probe_rates(void* stream, double* out) {
    using namespace kpcg;
    try {
        if (!out) fail(KPCG_ERR_ARG, "out is NULL");
        int dev = 0, sms = 0;
        KPCG_CUDA(cudaGetDevice(&dev));
        KPCG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        cudaStream_t st = (cudaStream_t)stream;
        DevBuf<float> sink;
        DevBuf<unsigned long long> clk;
        float* s = sink.need(kThreads);
        unsigned long long* c = clk.need(2);
        double mhz[3];
        out[0] = probe_one<0>(sms, st, s, c, &mhz[0]);
        out[1] = probe_one<1>(sms, st, s, c, &mhz[1]);
        out[2] = probe_one<2>(sms, st, s, c, &mhz[2]);
        out[3] = mhz[0];
        out[4] = mhz[1];
        out[5] = mhz[2];
        out[6] = (double)sms;
        return KPCG_OK;
    } catch (const Error& e) {
        set_handleless_error(e.msg);
        return e.status;
    }
}
