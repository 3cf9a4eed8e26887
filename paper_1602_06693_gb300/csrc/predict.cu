// Predictions at test inputs (Sec. 2.1: the predictive mean and variance need
// the same kernel products as training, and the variance one linear system
// per test point; Sec. 5 scores both):
//     m_* = K(X_*, X) alpha,        v_* = s^2 - k_*^T K_y^{-1} k_*,
// with k_* = K(X, x_*) (the latent variance; add sigma^2 for a noisy target).
// The mean is a rectangular FP64 product with entries rebuilt from the scaled
// inputs (nothing n x n_* stored); the variance solves blocks of up to 16
// test points as right-hand sides with the handle's own solver, then reduces
// v_* = s^2 - k_*^T w_* in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "solver.cuh"

namespace kpcg {
namespace {

constexpr int PT = 256;   // threads per CTA
constexpr int PJ = 64;    // training rows per shared-memory tile
constexpr int PB = 16;    // test points per variance block

// x'_* = (x_* - mu) / l * sqrt(1/2), zero-padded to dp (the training scaling).
__global__ void pred_prescale_kernel(const float* __restrict__ Xs, int64_t ns, int d, int dp,
                                     const double* __restrict__ mu,
                                     const double* __restrict__ inv_ell,
                                     double* __restrict__ xt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ns * dp) return;
    const int64_t i = e / dp;
    const int q = (int)(e - i * dp);
    xt[e] = (q < d) ? ((double)Xs[i * d + q] - mu[q]) * inv_ell[q] * 0.70710678118654752440 : 0.0;
}

// part[split][i] = sum_{j in split} s^2 exp(-|x'_*i - x'_j|^2) alpha_j (FP64,
// direct differences); one test point per thread.
template <int DP>
__global__ void __launch_bounds__(PT)
    pred_mean_kernel(const double* __restrict__ xt, int64_t ns, const double* __restrict__ xs,
                     int64_t n, double c0, const double* __restrict__ alpha, int64_t cps,
                     double* __restrict__ part) {
    __shared__ double sx[PJ * DP];
    __shared__ double sa[PJ];
    const int64_t i = (int64_t)blockIdx.x * PT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * cps;
    const int64_t j1 = min(n, j0 + cps);
    double xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < ns) ? xt[i * DP + q] : 0.0;
    double acc = 0.0;
    for (int64_t jt = j0; jt < j1; jt += PJ) {
        const int jn = (int)min((int64_t)PJ, j1 - jt);
        __syncthreads();
        for (int e = threadIdx.x; e < PJ * DP; e += PT)
            sx[e] = (e / DP < jn) ? xs[jt * DP + e] : 0.0;
        for (int e = threadIdx.x; e < PJ; e += PT) sa[e] = (e < jn) ? alpha[jt + e] : 0.0;
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            double a = c0;
#pragma unroll
            for (int q = 0; q < DP; ++q) {
                const double t = xi[q] - sx[jj * DP + q];
                a = fma(-t, t, a);
            }
            acc = fma(exp(a), sa[jj], acc);
        }
    }
    if (i < ns) part[(int64_t)blockIdx.y * ns + i] = acc;
}

__global__ void pred_mean_reduce_kernel(const double* __restrict__ part, int nsplit, int64_t ns,
                                        double* __restrict__ mean) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * ns + i];
    mean[i] = s;
}

// K[i][b] = s^2 exp(-|x'_i - x'_*b|^2): the right-hand sides k_* of one block.
__global__ void pred_kblock_kernel(const double* __restrict__ xs, int64_t n, int dp,
                                   const double* __restrict__ xt, double c0, double* __restrict__ K,
                                   int64_t ldk) {
    const int b = blockIdx.y;
    const double* xb = xt + (int64_t)b * dp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double a = c0;
        for (int q = 0; q < dp; ++q) {
            const double t = xs[i * dp + q] - xb[q];
            a = fma(-t, t, a);
        }
        K[i + (int64_t)b * ldk] = exp(a);
    }
}

template <int DP>
void launch_mean(const double* xt, int64_t ns, const double* xs, int64_t n, double c0,
                 const double* alpha, int64_t cps, int nsplit, double* part, cudaStream_t st) {
    dim3 g((unsigned)((ns + PT - 1) / PT), (unsigned)nsplit);
    pred_mean_kernel<DP><<<g, PT, 0, st>>>(xt, ns, xs, n, c0, alpha, cps, part);
    KPCG_LAUNCHED("pred_mean_kernel");
}

}  // namespace

const double* predict_mean(Ctx& c, const float* Xs, int64_t ns, const double* alpha,
                           double* mean) {
    cudaStream_t st = c.stream;
    const int dp = c.dp;
    const double c0 = c.c0_64();
    double* xt = c.pxt.need((size_t)ns * dp);
    pred_prescale_kernel<<<(unsigned)((ns * dp + 255) / 256), 256, 0, st>>>(
        Xs, ns, c.d, dp, c.mu.p, c.inv_ell.p, xt);
    KPCG_LAUNCHED("pred_prescale_kernel");
    // column ranges split over about eight CTAs per SM, added in order
    const int64_t nrb = (ns + PT - 1) / PT;
    int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((152 * 8 + nrb - 1) / nrb,
                                                            (c.n + PJ - 1) / PJ));
    int64_t cps = ((c.n + nsplit - 1) / nsplit + PJ - 1) / PJ * PJ;
    nsplit = (c.n + cps - 1) / cps;
    double* part = c.ppart.need((size_t)nsplit * ns);
    switch (dp) {
        case 4: launch_mean<4>(xt, ns, c.xs64.p, c.n, c0, alpha, cps, (int)nsplit, part, st); break;
        case 8: launch_mean<8>(xt, ns, c.xs64.p, c.n, c0, alpha, cps, (int)nsplit, part, st); break;
        case 12: launch_mean<12>(xt, ns, c.xs64.p, c.n, c0, alpha, cps, (int)nsplit, part, st); break;
        case 16: launch_mean<16>(xt, ns, c.xs64.p, c.n, c0, alpha, cps, (int)nsplit, part, st); break;
        case 32: launch_mean<32>(xt, ns, c.xs64.p, c.n, c0, alpha, cps, (int)nsplit, part, st); break;
        default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
    }
    pred_mean_reduce_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(part, (int)nsplit, ns,
                                                                          mean);
    KPCG_LAUNCHED("pred_mean_reduce_kernel");
    return xt;
}

void predict_kblock(Ctx& c, const double* xt, int nb, double* Kb, int64_t ldk) {
    pred_kblock_kernel<<<dim3((unsigned)std::min<int64_t>((c.n + 255) / 256, 512), (unsigned)nb),
                         256, 0, c.stream>>>(c.xs64.p, c.n, c.dp, xt, c.c0_64(), Kb, ldk);
    KPCG_LAUNCHED("pred_kblock_kernel");
}

}  // namespace kpcg

using kpcg::fail;

extern "C" {

kpcg_status kpcg_predict(kpcg_t h, const float* Xs, int64_t ns, const double* alpha,
                         double* mean, double* var, double tol, kpcg_info* info) {
    if (!h) return KPCG_ERR_ARG;
    try {
        using namespace kpcg;
        if (ns < 0) fail(KPCG_ERR_ARG, "ns must be >= 0");
        if (ns == 0) return KPCG_OK;
        if (!Xs || !alpha || !mean) fail(KPCG_ERR_ARG, "NULL argument");
        if (var && !(tol > 0.0)) fail(KPCG_ERR_ARG, "tol must be > 0");
        Ctx& c = *h;
        cudaStream_t st = c.stream;
        const int dp = c.dp;
        const double* xt = predict_mean(c, Xs, ns, alpha, mean);
        kpcg_info tot{};
        double max_rel = 0.0;
        if (var) {
            // one solve per block of up to 16 test points (Sec. 2.1)
            const int64_t ld = c.ld;
            double* Kb = c.pKb.need((size_t)ld * PB);
            double* W = c.pW.need((size_t)ld * PB);
            std::vector<double> hv((size_t)ns);
            const int nblk = dot_blocks(c.n);
            for (int64_t b0 = 0; b0 < ns; b0 += PB) {
                const int nb = (int)std::min<int64_t>(PB, ns - b0);
                predict_kblock(c, xt + b0 * dp, nb, Kb, ld);
                kpcg_info bi{};
                const kpcg_status s = solve_impl(c, Kb, ld, nb, tol, nullptr, W, ld, nullptr, &bi);
                if (s != KPCG_OK) fail(s, "variance solve: " + c.err);
                tot.iters_total += bi.iters_total;
                tot.outer_steps += bi.outer_steps;
                tot.launches += bi.launches;
                tot.kv_inner_ms += bi.kv_inner_ms;
                tot.kv_inner_calls += bi.kv_inner_calls;
                tot.kv_outer_ms += bi.kv_outer_ms;
                tot.kv_outer_calls += bi.kv_outer_calls;
                tot.precond_ms += bi.precond_ms;
                tot.precond_calls += bi.precond_calls;
                max_rel = std::max(max_rel, bi.max_rel_res);
                double* pp = c.partial.need((size_t)nblk * nb);
                dot_cols<double>(Kb, ld, W, ld, c.n, nb, pp, nblk, st);
                std::vector<double> hp((size_t)nblk * nb);
                KPCG_CUDA(cudaMemcpyAsync(hp.data(), pp, sizeof(double) * hp.size(),
                                          cudaMemcpyDeviceToHost, st));
                KPCG_CUDA(cudaStreamSynchronize(st));
                for (int k = 0; k < nb; ++k) {
                    double q = 0.0;
                    for (int t = 0; t < nblk; ++t) q += hp[(size_t)k * nblk + t];
                    hv[(size_t)(b0 + k)] = c.s2 - q;
                }
            }
            KPCG_CUDA(cudaMemcpyAsync(var, hv.data(), sizeof(double) * ns,
                                      cudaMemcpyHostToDevice, st));
        }
        KPCG_CUDA(cudaStreamSynchronize(st));
        if (info) {
            *info = tot;
            info->max_rel_res = max_rel;
        }
        return KPCG_OK;
    } catch (const kpcg::Error& e) {
        h->err = e.msg;
        return e.status;
    }
}

}  // extern "C"
