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
constexpr double kRebuildDrift = 0.1;  // relative drift of W^1/2 that rebuilds P_B

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

// dst = s * src (element-wise in T), c columns.
template <typename T>
__global__ void lap_scale_kernel(T* __restrict__ dst, int64_t ldd, const T* __restrict__ src,
                                 int64_t lds, const T* __restrict__ s, int64_t n) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i + k * ldd] = s[i] * src[i + k * lds];
}

// out = p + s * u (the last step of the B product), c columns.
template <typename T>
__global__ void lap_bfinish_kernel(T* out, int64_t ldo, const T* __restrict__ p, int64_t ldp,
                                   const T* u, int64_t ldu, const T* __restrict__ s, int64_t n) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i + k * ldo] = fma(s[i], u[i + k * ldu], p[i + k * ldp]);
}

// s32 = (float) s
__global__ void lap_to_f32_kernel(float* __restrict__ d, const double* __restrict__ s,
                                  int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}

// r = v - w, c columns of leading dimension ld
__global__ void lap_sub_kernel(double* __restrict__ r, const double* __restrict__ v,
                               const double* __restrict__ w, int64_t n, int64_t ld) {
    const int64_t o = (int64_t)blockIdx.y * ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        r[o + i] = v[o + i] - w[o + i];
}

// p_* = Phi(m_* / sqrt(1 + v_*)), the probit predictive probability
__global__ void lap_prob_kernel(const double* __restrict__ m, const double* __restrict__ v,
                                int64_t ns, double* __restrict__ prob) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) prob[i] = normcdf(m[i] / sqrt(1.0 + v[i]));
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

// part[blk] = max_i |sW_i / sWb_i - 1| over the block's rows (the drift of W^1/2
// since the preconditioner of B was built on sWb)
__global__ void __launch_bounds__(256)
    lap_drift_kernel(const double* __restrict__ sW, const double* __restrict__ sWb, int64_t n,
                     double* __restrict__ part) {
    __shared__ double sm[256];
    double mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        mx = fmax(mx, fabs(sW[i] / sWb[i] - 1.0));
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
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

// B P = P + sW (K (sW P)) for up to the scratch width of columns: w = sW P,
// u = K w (double-float), then the sum.  Launches on H.stream at call time
// (graph capture swaps it).
VecOp make_bop(Ctx* hp, const double* sW, double* u, double* w) {
    return [hp, sW, u, w](const double* P, int64_t ldp, int cc, double* Q, int64_t ldq) {
        Ctx& H = *hp;
        const dim3 gg(lap_grid(H.n), (unsigned)cc);
        lap_scale_kernel<double><<<gg, 256, 0, H.stream>>>(w, H.ld, P, ldp, sW, H.n);
        KPCG_LAUNCHED("lap_scale_kernel");
        kv_df(H, w, H.ld, cc, nullptr, 0, u, H.ld, 0.0);
        lap_bfinish_kernel<double><<<gg, 256, 0, H.stream>>>(Q, ldq, P, ldp, u, H.ld, sW, H.n);
        KPCG_LAUNCHED("lap_bfinish_kernel");
    };
}

// The preconditioner of B: the Nystrom form in H.LP, or the identity.
VecOp make_bpc(Ctx* hp, bool pre) {
    return [hp, pre](const double* R, int64_t ldr, int cc, double* Z, int64_t ldz) {
        Ctx& H = *hp;
        if (pre)
            precond_apply_f64(H.LP, R, ldr, cc, Z, ldz, H.stream);
        else
            copy_cols<double>(Z, ldz, R, ldr, H.n, cc, H.stream);
    };
}

// B Z = R for nb columns (ld-strided): PCG from zero (from Z if z_given), then each column's
// residual is recomputed with a fresh product and CG restarts from Z while
// one misses tol (at most 4 restarts).  t, r: scratch of nb columns.  Adds
// the iterations (the most any column took) to cg_total; returns the worst
// certified relative residual.
double bsolve(Ctx& c, const VecOp& mvB, const VecOp& pcB, const double* R, int nb, double* Z,
              double tol, double* t, double* r, int& cg_total, bool z_given = false) {
    const int64_t n = c.n, ld = c.ld;
    const int nblk = dot_blocks(n);
    std::vector<int> iters;
    double worst = 0.0;
    for (int attempt = 0; attempt < 5; ++attempt) {
        int broken = 0;
        pcg_f64(c, nb, R, ld, Z, ld, attempt == 0 && !z_given, tol, c.opt.max_iter, mvB, pcB,
                c.lcg, iters, broken);
        cg_total += iters.empty() ? 0 : *std::max_element(iters.begin(), iters.end());
        if (broken) fail(KPCG_ERR_BREAKDOWN, "breakdown in a B-solve");
        mvB(Z, ld, nb, t, ld);
        lap_sub_kernel<<<dim3(lap_grid(n), (unsigned)nb), 256, 0, c.stream>>>(r, R, t, n, ld);
        KPCG_LAUNCHED("lap_sub_kernel");
        double* pp = c.partial.need((size_t)nblk * nb * 2);
        dot_cols<double>(r, ld, r, ld, n, nb, pp, nblk, c.stream);
        dot_cols<double>(R, ld, R, ld, n, nb, pp + (size_t)nblk * nb, nblk, c.stream);
        std::vector<double> hq((size_t)nblk * nb * 2);
        KPCG_CUDA(cudaMemcpyAsync(hq.data(), pp, sizeof(double) * hq.size(),
                                  cudaMemcpyDeviceToHost, c.stream));
        KPCG_CUDA(cudaStreamSynchronize(c.stream));
        worst = 0.0;
        for (int k = 0; k < nb; ++k) {
            double rr = 0.0, vv = 0.0;
            for (int q = 0; q < nblk; ++q) {
                rr += hq[(size_t)k * nblk + q];
                vv += hq[(size_t)(nb + k) * nblk + q];
            }
            worst = std::max(worst, vv > 0.0 ? std::sqrt(rr / vv) : 0.0);
        }
        if (worst <= tol) break;
    }
    return worst;
}

// Scratch of the mixed-precision B-solve: FP32 W^1/2 and two FP32 blocks.
struct LapMixed {
    const float* sW32;
    float *w32, *u32;
};

// The B operators for the flexible-CG solve of fcg_solve: inner FP32 products
// B v = v + sW (K (sW v)) with the tensor-core (tc) or FP32 K.V and the FP32
// apply of P_B; outer products and every residual with the double-float B
// product (B >= I, so a residual of FP64 class certifies it).  r is scratch.
MixedOps lap_mixed_ops(Ctx* hp, const VecOp& mvB, const LapMixed& m, bool tc, bool pre,
                       double* r) {
    MixedOps o;
    o.inner_mv = [hp, m, tc](const float* V, int64_t ldv, int cc, float* O, int64_t ldo) {
        Ctx& H = *hp;
        const dim3 gg(lap_grid(H.n), (unsigned)cc);
        lap_scale_kernel<float><<<gg, 256, 0, H.stream>>>(m.w32, H.ld, V, ldv, m.sW32, H.n);
        KPCG_LAUNCHED("lap_scale_kernel");
        if (tc)
            kv_tc_inner(H, m.w32, H.ld, cc, m.u32, H.ld, 0.f);
        else
            kv_f32(H.xs32.p, H.n, H.dp, H.c0_32(), 0.f, m.w32, H.ld, cc, m.u32, H.ld, H.kvws,
                   H.stream);
        lap_bfinish_kernel<float><<<gg, 256, 0, H.stream>>>(O, ldo, V, ldv, m.u32, H.ld, m.sW32,
                                                            H.n);
        KPCG_LAUNCHED("lap_bfinish_kernel");
    };
    o.inner_pc = [hp, pre](const float* R, int64_t ldr, int cc, float* Z, int64_t ldz) {
        Ctx& H = *hp;
        if (pre)
            precond_apply_f32(H.LP, R, ldr, cc, Z, ldz, H.stream);
        else
            copy_cols<float>(Z, ldz, R, ldr, H.n, cc, H.stream);
    };
    o.outer_mv = mvB;
    o.residual = [hp, mvB, r](const double* B, int64_t ldb, int cc, const double* X, int64_t ldx,
                              double* R, std::vector<double>& rr, std::vector<double>& bb,
                              bool) {
        Ctx& H = *hp;
        if (ldb != H.ld) fail(KPCG_ERR_ARG, "B-solve right-hand sides must have leading dim ld");
        mvB(X, ldx, cc, r, H.ld);
        lap_sub_kernel<<<dim3(lap_grid(H.n), (unsigned)cc), 256, 0, H.stream>>>(R, B, r, H.n,
                                                                                 H.ld);
        KPCG_LAUNCHED("lap_sub_kernel");
        const int nblk = dot_blocks(H.n);
        double* pp = H.partial.need((size_t)nblk * cc * 2);
        dot_cols<double>(R, H.ld, R, H.ld, H.n, cc, pp, nblk, H.stream);
        dot_cols<double>(B, ldb, B, ldb, H.n, cc, pp + (size_t)nblk * cc, nblk, H.stream);
        std::vector<double> hq((size_t)nblk * cc * 2);
        KPCG_CUDA(cudaMemcpyAsync(hq.data(), pp, sizeof(double) * hq.size(),
                                  cudaMemcpyDeviceToHost, H.stream));
        KPCG_CUDA(cudaStreamSynchronize(H.stream));
        rr.assign((size_t)cc, 0.0);
        bb.assign((size_t)cc, 0.0);
        for (int k = 0; k < cc; ++k)
            for (int q = 0; q < nblk; ++q) {
                rr[(size_t)k] += hq[(size_t)k * nblk + q];
                bb[(size_t)k] += hq[(size_t)(cc + k) * nblk + q];
            }
    };
    if (tc) o.timed_out = [hp]() { return kv_tc_error(*hp) != 0; };
    return o;
}

// B Z = R (nb columns, leading dimension ld): with a mixed operator set, the
// flexible-CG solve (from Z if z_given; tol_mode forced to the relative test),
// else bsolve.  Returns the worst certified relative residual.
double solve_b(Ctx& c, const VecOp& mvB, const VecOp& pcB, const MixedOps* mixed,
               const double* R, int nb, double* Z, double tol, double* t, double* r,
               int& cg_total, bool z_given) {
    if (!mixed) return bsolve(c, mvB, pcB, R, nb, Z, tol, t, r, cg_total, z_given);
    std::vector<int> iters_col((size_t)nb, 0);
    int iters_total = 0, steps = 0;
    std::vector<double> rr, bb;
    const int saved_mode = c.opt.tol_mode;
    c.opt.tol_mode = 0;
    kpcg_status stt;
    try {
        stt = fcg_solve(c, *mixed, R, c.ld, nb, tol, z_given ? Z : nullptr, Z, c.ld, iters_col,
                        iters_total, steps, rr, bb);
    } catch (...) {
        c.opt.tol_mode = saved_mode;
        throw;
    }
    c.opt.tol_mode = saved_mode;
    cg_total += iters_total;
    if (stt == KPCG_ERR_BREAKDOWN) fail(KPCG_ERR_BREAKDOWN, "breakdown in a B-solve");
    double worst = 0.0;
    for (int k = 0; k < nb && k < (int)rr.size(); ++k)
        if (bb[(size_t)k] > 0.0) worst = std::max(worst, std::sqrt(rr[(size_t)k] / bb[(size_t)k]));
    return worst;
}

void check_labels(Ctx& c, const double* y) {
    std::vector<double> hy((size_t)c.n);
    KPCG_CUDA(cudaMemcpyAsync(hy.data(), y, sizeof(double) * c.n, cudaMemcpyDeviceToHost,
                              c.stream));
    KPCG_CUDA(cudaStreamSynchronize(c.stream));
    for (double v : hy)
        if (v != 1.0 && v != -1.0) fail(KPCG_ERR_ARG, "labels must be +1 or -1");
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
        check_labels(c, y);
        // vectors f, a, sW = W^1/2, b, v, z, sWb (sW of the last P_B build); u, w,
        // t, r are scratch of the B-solve
        double* base = c.lap.need((size_t)ld * 11 + 2 * 152 * 8);
        double* f = base;
        double* a = base + ld;
        double* sW = base + 2 * ld;
        double* b = base + 3 * ld;
        double* v = base + 4 * ld;
        double* z = base + 5 * ld;
        double* u = base + 6 * ld;
        double* w = base + 7 * ld;
        double* t = base + 8 * ld;
        double* r = base + 9 * ld;
        double* sWb = base + 10 * ld;
        double* part = base + 11 * ld;
        KPCG_CUDA(cudaMemsetAsync(f, 0, sizeof(double) * ld, st));
        KPCG_CUDA(cudaMemsetAsync(a, 0, sizeof(double) * ld, st));
        const unsigned g = lap_grid(n);
        const bool pre = c.pkind == KPCG_PREC_NYSTROM;
        const VecOp mvB = make_bop(&c, sW, u, w);
        const VecOp pcB = make_bpc(&c, pre);
        // mixed precision (KPCG_TC_IR / KPCG_FP32_IR): FP32 W^1/2 and scratch
        const bool tc = c.opt.precision == KPCG_TC_IR;
        const bool use_mixed = tc || c.opt.precision == KPCG_FP32_IR;
        if (tc && !kv_tc_supported(c.d))
            fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
        float* f32 = c.lpw32.need((size_t)ld * 3);
        const LapMixed lm{f32, f32 + ld, f32 + 2 * ld};
        MixedOps mops;
        if (use_mixed) mops = lap_mixed_ops(&c, mvB, lm, tc, pre, t);
        const MixedOps* mixed = use_mixed ? &mops : nullptr;

        double psi_old = lap_psi(c, y, f, a, part);  // n log(1/2) at f = 0
        double psi = psi_old, setup_ms = 0.0, worst = 0.0;
        int steps = 0, cg_total = 0, builds = 0;
        bool converged = false, solved = true;
        while (steps < max_newton) {
            ++steps;
            lap_terms_kernel<<<g, 256, 0, st>>>(y, f, n, sW, b);
            KPCG_LAUNCHED("lap_terms_kernel");
            // P_B is rebuilt when W^1/2 moved by more than 10% on some row since
            // the last build; a stale P_B is still SPD, so PCG stays correct
            bool rebuild = pre && builds == 0;
            if (pre && builds > 0) {
                lap_drift_kernel<<<g, 256, 0, st>>>(sW, sWb, n, part);
                KPCG_LAUNCHED("lap_drift_kernel");
                std::vector<double> hd(g);
                KPCG_CUDA(cudaMemcpyAsync(hd.data(), part, sizeof(double) * g,
                                          cudaMemcpyDeviceToHost, st));
                KPCG_CUDA(cudaStreamSynchronize(st));
                rebuild = *std::max_element(hd.begin(), hd.end()) > kRebuildDrift;
            }
            if (rebuild) {
                ++builds;
                KPCG_CUDA(cudaMemcpyAsync(sWb, sW, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                          st));
                const auto s0 = std::chrono::steady_clock::now();
                laplace_precond_setup(c.LP, c.lkxu0, builds == 1, c.xs32.p, c.xs64.p, n, c.dp,
                                      c.c0_64(), sW, c.pidx.data(), c.psize, st);
                KPCG_CUDA(cudaStreamSynchronize(st));
                setup_ms += std::chrono::duration<double, std::milli>(
                                std::chrono::steady_clock::now() - s0)
                                .count();
            }
            // v = sW (K b)
            kv_df(c, b, ld, 1, nullptr, 0, u, ld, 0.0);
            lap_scale_kernel<double><<<dim3(g, 1), 256, 0, st>>>(v, ld, u, ld, sW, n);
            KPCG_LAUNCHED("lap_scale_kernel");
            // from the previous step's z: B and v change little near the mode
            if (use_mixed) {
                lap_to_f32_kernel<<<g, 256, 0, st>>>(f32, sW, n);
                KPCG_LAUNCHED("lap_to_f32_kernel");
            }
            const double rel =
                solve_b(c, mvB, pcB, mixed, v, 1, z, cg_tol, t, r, cg_total, steps > 1);
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
            info->precond_builds = builds;
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

kpcg_status kpcg_laplace_predict(kpcg_t h, const double* y, const double* f, const double* a,
                                 const float* Xs, int64_t ns, double* mean, double* var,
                                 double* prob, double cg_tol, kpcg_laplace_info* info) {
    if (!h) return KPCG_ERR_ARG;
    try {
        using namespace kpcg;
        Ctx& c = *h;
        const auto t0 = std::chrono::steady_clock::now();
        const long long launches0 = launch_count();
        if (ns < 0) fail(KPCG_ERR_ARG, "ns must be >= 0");
        if (ns == 0) return KPCG_OK;
        if (!y || !f || !a || !Xs || !mean) fail(KPCG_ERR_ARG, "NULL argument");
        const bool want_var = var || prob;
        if (want_var && !(cg_tol > 0.0 && cg_tol < 1.0))
            fail(KPCG_ERR_ARG, "cg_tol must be in (0, 1)");
        if (c.pkind != KPCG_PREC_NONE && c.pkind != KPCG_PREC_NYSTROM)
            fail(KPCG_ERR_ARG, "the Laplace B-solve takes a Nystrom preconditioner or none");
        cudaStream_t st = c.stream;
        check_labels(c, y);
        // latent mean m_* = K(X_*, X) a
        const double* xt = predict_mean(c, Xs, ns, a, mean);
        int cg_total = 0, pre_built = 0;
        double worst = 0.0, setup_ms = 0.0;
        bool solved = true;
        if (want_var) {
            constexpr int PB = 16;  // test points per block of right-hand sides
            const int64_t n = c.n, ld = c.ld;
            double* base = c.lpw.need((size_t)ld * (2 + 7 * PB));
            double* sW = base;
            double* bb = base + ld;
            double* Kb = base + 2 * ld;
            double* R = Kb + PB * ld;
            double* Z = R + PB * ld;
            double* u = Z + PB * ld;
            double* w = u + PB * ld;
            double* t = w + PB * ld;
            double* r = t + PB * ld;
            const unsigned g = lap_grid(n);
            lap_terms_kernel<<<g, 256, 0, st>>>(y, f, n, sW, bb);  // W at the mode
            KPCG_LAUNCHED("lap_terms_kernel");
            const bool pre = c.pkind == KPCG_PREC_NYSTROM;
            if (pre) {
                const auto s0 = std::chrono::steady_clock::now();
                laplace_precond_setup(c.LP, c.lkxu0, true, c.xs32.p, c.xs64.p, n, c.dp,
                                      c.c0_64(), sW, c.pidx.data(), c.psize, st);
                pre_built = 1;
                KPCG_CUDA(cudaStreamSynchronize(st));
                setup_ms = std::chrono::duration<double, std::milli>(
                               std::chrono::steady_clock::now() - s0)
                               .count();
            }
            const VecOp mvB = make_bop(&c, sW, u, w);
            const VecOp pcB = make_bpc(&c, pre);
            const bool tc = c.opt.precision == KPCG_TC_IR;
            const bool use_mixed = tc || c.opt.precision == KPCG_FP32_IR;
            if (tc && !kv_tc_supported(c.d))
                fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
            float* f32 = c.lpw32.need((size_t)ld * (1 + 2 * PB));
            const LapMixed lm{f32, f32 + ld, f32 + (1 + PB) * ld};
            MixedOps mops;
            if (use_mixed) {
                lap_to_f32_kernel<<<g, 256, 0, st>>>(f32, sW, n);
                KPCG_LAUNCHED("lap_to_f32_kernel");
                mops = lap_mixed_ops(&c, mvB, lm, tc, pre, t);
            }
            const MixedOps* mixed = use_mixed ? &mops : nullptr;
            const int nblk = dot_blocks(n);
            std::vector<double> hv((size_t)ns);
            for (int64_t b0 = 0; b0 < ns; b0 += PB) {
                const int nb = (int)std::min<int64_t>(PB, ns - b0);
                // R = W^1/2 k_*, Z = B^{-1} R, v_* = s^2 - R^T Z
                predict_kblock(c, xt + b0 * c.dp, nb, Kb, ld);
                lap_scale_kernel<double><<<dim3(g, (unsigned)nb), 256, 0, st>>>(R, ld, Kb, ld, sW,
                                                                                n);
                KPCG_LAUNCHED("lap_scale_kernel");
                const double rel =
                    solve_b(c, mvB, pcB, mixed, R, nb, Z, cg_tol, t, r, cg_total, false);
                worst = std::max(worst, rel);
                if (rel > cg_tol) solved = false;
                double* pp = c.partial.need((size_t)nblk * nb);
                dot_cols<double>(R, ld, Z, ld, n, nb, pp, nblk, st);
                std::vector<double> hp((size_t)nblk * nb);
                KPCG_CUDA(cudaMemcpyAsync(hp.data(), pp, sizeof(double) * hp.size(),
                                          cudaMemcpyDeviceToHost, st));
                KPCG_CUDA(cudaStreamSynchronize(st));
                for (int k = 0; k < nb; ++k) {
                    double q = 0.0;
                    for (int e = 0; e < nblk; ++e) q += hp[(size_t)k * nblk + e];
                    hv[(size_t)(b0 + k)] = c.s2 - q;
                }
            }
            double* vd = var ? var : c.lpv.need((size_t)ns);
            KPCG_CUDA(cudaMemcpyAsync(vd, hv.data(), sizeof(double) * ns, cudaMemcpyHostToDevice,
                                      st));
            if (prob) {
                lap_prob_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(mean, vd, ns, prob);
                KPCG_LAUNCHED("lap_prob_kernel");
            }
        }
        KPCG_CUDA(cudaStreamSynchronize(st));
        if (info) {
            info->newton_steps = 0;
            info->precond_builds = pre_built;
            info->cg_iters_total = cg_total;
            info->psi = 0.0;
            info->max_rel_res = worst;
            info->setup_ms = setup_ms;
            info->time_ms = std::chrono::duration<double, std::milli>(
                                std::chrono::steady_clock::now() - t0)
                                .count();
            info->launches = (int)(launch_count() - launches0);
        }
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
