// GP classification with the probit likelihood: the Newton iteration of the
// Laplace approximation (Sec. 2.2; Appendix B, Algorithm "Laplace
// approximation for GPs").  Per step, with W = -d^2/df^2 log p(y|f) diagonal
// and g = d/df log p(y|f):
//     b = W f + g,   v = W^1/2 K b,   solve B z = v,   a = b - W^1/2 z,   f = K a,
// B = I + W^1/2 K W^1/2.  The two products with K and every product inside
// the B-solve are matrix-free (the double-float K.V); the per-point terms
// and all vector work are FP64.  Nothing n x n is stored.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "solver.cuh"

namespace kpcg {
namespace {

constexpr double kSqrt2OverPi = 0.79788456080286535588;  // sqrt(2 / pi)
constexpr double kSqrtHalf = 0.70710678118654752440;

// N(z) / Phi(z) for the standard normal density and CDF.  With
// Phi(z) = erfc(-z/sqrt2)/2 = erfcx(-z/sqrt2) exp(-z^2/2)/2 the exponentials
// cancel: r = sqrt(2/pi) / erfcx(-z/sqrt2), finite for every z.
__device__ __forceinline__ double probit_ratio(double z) {
    return kSqrt2OverPi / erfcx(-z * kSqrtHalf);
}

// log Phi(z): through erfcx below zero (no underflow of Phi), log1p above.
__device__ __forceinline__ double log_probit(double z) {
    if (z < 0.0) return log(0.5 * erfcx(-z * kSqrtHalf)) - 0.5 * z * z;
    return log1p(-0.5 * erfc(z * kSqrtHalf));
}

// Per point at the current f: z = y f, r = N(z)/Phi(z), g = y r,
// W = r^2 + z r (in (0, 1) for the probit likelihood), sW = W^1/2, b = W f + g.
__global__ void lap_terms_kernel(const double* __restrict__ y, const double* __restrict__ f,
                                 int64_t n, double* __restrict__ sW, double* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double yi = y[i], fi = f[i];
        const double z = yi * fi;
        const double r = probit_ratio(z);
        const double W = fma(r, r, z * r);
        sW[i] = sqrt(W);
        b[i] = fma(W, fi, yi * r);
    }
}

// dst = s * src (element-wise, FP64), c columns.
__global__ void lap_scale_kernel(double* __restrict__ dst, int64_t ldd,
                                 const double* __restrict__ src, int64_t lds,
                                 const double* __restrict__ s, int64_t n) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i + k * ldd] = s[i] * src[i + k * lds];
}

// out = p + s * u (the last step of the B product), c columns.
__global__ void lap_bfinish_kernel(double* out, int64_t ldo, const double* __restrict__ p,
                                   int64_t ldp, const double* u, int64_t ldu,
                                   const double* __restrict__ s, int64_t n) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i + k * ldo] = fma(s[i], u[i + k * ldu], p[i + k * ldp]);
}

// r = v - w
__global__ void lap_sub_kernel(double* __restrict__ r, const double* __restrict__ v,
                               const double* __restrict__ w, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        r[i] = v[i] - w[i];
}

// a = b - s * z
__global__ void lap_a_kernel(double* __restrict__ a, const double* __restrict__ b,
                             const double* __restrict__ s, const double* __restrict__ z,
                             int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = fma(-s[i], z[i], b[i]);
}

// Per block: sum of log Phi(y_i f_i) and of a_i f_i (fixed-order tree), into
// part[blk] and part[nblk + blk]; the host adds the blocks in order.
__global__ void __launch_bounds__(256)
    lap_psi_kernel(const double* __restrict__ y, const double* __restrict__ f,
                   const double* __restrict__ a, int64_t n, double* __restrict__ part) {
    __shared__ double s1[256], s2[256];
    double l = 0.0, q = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        l += log_probit(y[i] * f[i]);
        q = fma(a[i], f[i], q);
    }
    s1[threadIdx.x] = l;
    s2[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1[0];
        part[gridDim.x + blockIdx.x] = s2[0];
    }
}

unsigned lap_grid(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
}

// Psi = sum log Phi(y f) - 1/2 a^T f (FP64, deterministic order).
double lap_psi(Ctx& h, const double* y, const double* f, const double* a, double* part) {
    const unsigned g = lap_grid(h.n);
    lap_psi_kernel<<<g, 256, 0, h.stream>>>(y, f, a, h.n, part);
    KPCG_LAUNCHED("lap_psi_kernel");
    std::vector<double> hp((size_t)2 * g);
    KPCG_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost,
                              h.stream));
    KPCG_CUDA(cudaStreamSynchronize(h.stream));
    double l = 0.0, q = 0.0;
    for (unsigned b = 0; b < g; ++b) {
        l += hp[b];
        q += hp[g + b];
    }
    return l - 0.5 * q;
}

}  // namespace
}  // namespace kpcg

using kpcg::fail;

extern "C" {

kpcg_status kpcg_laplace(kpcg_t h, const double* y, double newton_tol, int32_t max_newton,
                         double cg_tol, double* f_out, double* a_out, kpcg_laplace_info* info) {
    if (!h) return KPCG_ERR_ARG;
    try {
        using namespace kpcg;
        Ctx& c = *h;
        const auto t0 = std::chrono::steady_clock::now();
        const long long launches0 = launch_count();
        if (!y || !f_out) fail(KPCG_ERR_ARG, "NULL argument");
        if (!(newton_tol > 0.0)) fail(KPCG_ERR_ARG, "newton_tol must be > 0");
        if (max_newton < 1) fail(KPCG_ERR_ARG, "max_newton must be >= 1");
        if (!(cg_tol > 0.0 && cg_tol < 1.0)) fail(KPCG_ERR_ARG, "cg_tol must be in (0, 1)");
        if (c.pkind != KPCG_PREC_NONE && c.pkind != KPCG_PREC_NYSTROM)
            fail(KPCG_ERR_ARG, "the Laplace B-solve takes a Nystrom preconditioner or none");
        const int64_t n = c.n, ld = c.ld;
        cudaStream_t st = c.stream;
        {
            std::vector<double> hy((size_t)n);
            KPCG_CUDA(cudaMemcpyAsync(hy.data(), y, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                      st));
            KPCG_CUDA(cudaStreamSynchronize(st));
            for (double v : hy)
                if (v != 1.0 && v != -1.0) fail(KPCG_ERR_ARG, "labels must be +1 or -1");
        }
        // vectors f, a, sW = W^1/2, b, v, z; u and w are scratch of the B product
        double* base = c.lap.need((size_t)ld * 8 + 2 * 152 * 8);
        double* f = base;
        double* a = base + ld;
        double* sW = base + 2 * ld;
        double* b = base + 3 * ld;
        double* v = base + 4 * ld;
        double* z = base + 5 * ld;
        double* u = base + 6 * ld;
        double* w = base + 7 * ld;
        double* part = base + 8 * ld;
        KPCG_CUDA(cudaMemsetAsync(f, 0, sizeof(double) * ld, st));
        KPCG_CUDA(cudaMemsetAsync(a, 0, sizeof(double) * ld, st));
        const unsigned g = lap_grid(n);
        const bool pre = c.pkind == KPCG_PREC_NYSTROM;

        // B p = p + sW (K (sW p)), on h.stream at call time (graph capture swaps it)
        Ctx* hp = &c;
        const VecOp mvB = [hp, sW, u, w](const double* P, int64_t ldp, int cc, double* Q,
                                         int64_t ldq) {
            Ctx& H = *hp;
            const dim3 gg(lap_grid(H.n), (unsigned)cc);
            lap_scale_kernel<<<gg, 256, 0, H.stream>>>(w, H.ld, P, ldp, sW, H.n);
            KPCG_LAUNCHED("lap_scale_kernel");
            kv_df(H, w, H.ld, cc, nullptr, 0, u, H.ld, 0.0);
            lap_bfinish_kernel<<<gg, 256, 0, H.stream>>>(Q, ldq, P, ldp, u, H.ld, sW, H.n);
            KPCG_LAUNCHED("lap_bfinish_kernel");
        };
        const VecOp pcB = [hp, pre](const double* R, int64_t ldr, int cc, double* Z, int64_t ldz) {
            Ctx& H = *hp;
            if (pre)
                precond_apply_f64(H.LP, R, ldr, cc, Z, ldz, H.stream);
            else
                copy_cols<double>(Z, ldz, R, ldr, H.n, cc, H.stream);
        };

        double psi_old = lap_psi(c, y, f, a, part);  // n log(1/2) at f = 0
        double psi = psi_old, setup_ms = 0.0, worst = 0.0;
        int steps = 0, cg_total = 0;
        bool converged = false, solved = true;
        std::vector<int> iters;
        const int nblk = dot_blocks(n);
        while (steps < max_newton) {
            ++steps;
            lap_terms_kernel<<<g, 256, 0, st>>>(y, f, n, sW, b);
            KPCG_LAUNCHED("lap_terms_kernel");
            if (pre) {
                const auto s0 = std::chrono::steady_clock::now();
                laplace_precond_setup(c.LP, c.lkxu0, steps == 1, c.xs32.p, c.xs64.p, n, c.dp,
                                      c.c0_64(), sW, c.pidx.data(), c.psize, st);
                KPCG_CUDA(cudaStreamSynchronize(st));
                setup_ms += std::chrono::duration<double, std::milli>(
                                std::chrono::steady_clock::now() - s0)
                                .count();
            }
            // v = sW (K b)
            kv_df(c, b, ld, 1, nullptr, 0, u, ld, 0.0);
            lap_scale_kernel<<<dim3(g, 1), 256, 0, st>>>(v, ld, u, ld, sW, n);
            KPCG_LAUNCHED("lap_scale_kernel");
            // B z = v: PCG from zero; the recursive residual is re-certified with
            // a fresh product and CG restarts from z while it misses cg_tol
            double rel = 0.0;
            for (int attempt = 0; attempt < 5; ++attempt) {
                int broken = 0;
                pcg_f64(c, 1, v, ld, z, ld, attempt == 0, cg_tol, c.opt.max_iter, mvB, pcB,
                        c.lcg, iters, broken);
                cg_total += iters.empty() ? 0 : iters[0];
                if (broken) fail(KPCG_ERR_BREAKDOWN, "breakdown in the B-solve");
                // r = v - B z (w = B z; u, w are mvB's scratch, w written last)
                mvB(z, ld, 1, w, ld);
                lap_sub_kernel<<<g, 256, 0, st>>>(u, v, w, n);
                KPCG_LAUNCHED("lap_sub_kernel");
                double* pp = c.partial.need((size_t)nblk * 2);
                dot_cols<double>(u, ld, u, ld, n, 1, pp, nblk, st);
                dot_cols<double>(v, ld, v, ld, n, 1, pp + nblk, nblk, st);
                std::vector<double> hq((size_t)nblk * 2);
                KPCG_CUDA(cudaMemcpyAsync(hq.data(), pp, sizeof(double) * hq.size(),
                                          cudaMemcpyDeviceToHost, st));
                KPCG_CUDA(cudaStreamSynchronize(st));
                double rr = 0.0, vv = 0.0;
                for (int t = 0; t < nblk; ++t) {
                    rr += hq[(size_t)t];
                    vv += hq[(size_t)(nblk + t)];
                }
                rel = vv > 0.0 ? std::sqrt(rr / vv) : 0.0;
                if (rel <= cg_tol) break;
            }
            worst = std::max(worst, rel);
            if (rel > cg_tol) solved = false;
            // a = b - sW z;  f = K a
            lap_a_kernel<<<g, 256, 0, st>>>(a, b, sW, z, n);
            KPCG_LAUNCHED("lap_a_kernel");
            kv_df(c, a, ld, 1, nullptr, 0, f, ld, 0.0);
            psi = lap_psi(c, y, f, a, part);
            if (!std::isfinite(psi)) fail(KPCG_ERR_BREAKDOWN, "the Laplace objective is not finite");
            const bool done = std::fabs(psi - psi_old) <= newton_tol * std::max(1.0, std::fabs(psi));
            psi_old = psi;
            if (done) {
                converged = true;
                break;
            }
        }
        KPCG_CUDA(cudaMemcpyAsync(f_out, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        if (a_out)
            KPCG_CUDA(cudaMemcpyAsync(a_out, a, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        KPCG_CUDA(cudaStreamSynchronize(st));
        if (info) {
            info->newton_steps = steps;
            info->cg_iters_total = cg_total;
            info->psi = psi;
            info->max_rel_res = worst;
            info->setup_ms = setup_ms;
            info->time_ms = std::chrono::duration<double, std::milli>(
                                std::chrono::steady_clock::now() - t0)
                                .count();
            info->launches = (int)(launch_count() - launches0);
        }
        if (!converged) fail(KPCG_ERR_NO_CONVERGENCE, "Newton steps exhausted before the stop test");
        if (!solved) fail(KPCG_ERR_NO_CONVERGENCE, "a B-solve missed cg_tol");
        return KPCG_OK;
    } catch (const kpcg::Error& e) {
        h->err = e.msg;
        return e.status;
    } catch (const std::exception& e) {
        h->err = e.what();
        return KPCG_ERR_ARG;
    }
}

}  // extern "C"
