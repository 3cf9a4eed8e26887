// C ABI of libkpcg: handle life cycle, the batched PCG driver (Algorithm 1),
// mixed-precision refinement, and the stochastic gradient of Eq. 2.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kpcg_internal.cuh"
#include "ctx.cuh"
#include "precond.cuh"
#include "solver.cuh"

namespace kpcg {

[[noreturn]] void fail(kpcg_status s, const std::string& msg) { throw Error{s, msg}; }

void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
    if (e == cudaSuccess) return;
    const char* f = strrchr(file, '/');
    fail(e == cudaErrorMemoryAllocation ? KPCG_ERR_OOM : KPCG_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e) + " (" + (f ? f + 1 : file) + ":" +
             std::to_string(line) + ")");
}

static thread_local long long g_launches = 0;
void note_launch() { ++g_launches; }
void note_launches(long long k) { g_launches += k; }
bool trace_on() {
    static const int on = [] {
        const char* e = std::getenv("KPCG_TRACE");
        return (e && e[0] && e[0] != '0') ? 1 : 0;
    }();
    return on != 0;
}
long long launch_count() { return g_launches; }

int padded_dim(int d) {
    if (d <= 4) return 4;
    if (d <= 8) return 8;
    if (d <= 12) return 12;
    if (d <= 16) return 16;
    if (d <= 32) return 32;
    return -1;
}

namespace {

// Column means of X (FP64), one CTA per feature.
__global__ void colmean_kernel(const float* __restrict__ X, int64_t n, int d,
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

// x' = (x - mu) / l * g, zero-padded to dp columns; FP64 (g = sqrt(1/2)) and
// FP32 (g = sqrt(log2(e)/2)) copies.
__global__ void prescale_kernel(const float* __restrict__ X, int64_t n, int d, int dp,
                                const double* __restrict__ mu, const double* __restrict__ inv_ell,
                                double g64, double g32, double* __restrict__ xs64,
                                float* __restrict__ xs32) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * dp) return;
    const int64_t i = e / dp;
    const int q = (int)(e - i * dp);
    double v = 0.0;
    if (q < d) v = ((double)X[i * d + q] - mu[q]) * inv_ell[q];
    xs64[e] = v * g64;
    xs32[e] = (float)(v * g32);
}

template <typename T>
__global__ void sub_cols_t_kernel(T* __restrict__ R, int64_t ldr, const T* __restrict__ B,
                                  int64_t ldb, const T* __restrict__ Q, int64_t ldq, int64_t n) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        R[i + k * ldr] = B[i + k * ldb] - Q[i + k * ldq];
}

unsigned gx(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

}  // namespace

static thread_local std::string g_create_err;

// Message reported by kpcg_last_error(NULL) for calls that have no handle.
void set_handleless_error(const std::string& msg) { g_create_err = msg; }

static void ctx_rescale(Ctx& h) {
    std::vector<double> inv(h.d);
    for (int q = 0; q < h.d; ++q) {
        const double lt = h.ard ? h.log_theta[q] : h.log_theta[0];
        inv[q] = std::exp(-lt);
    }
    h.s2 = std::exp(h.log_theta.back());
    ++h.theta_version;
    KPCG_CUDA(cudaMemcpyAsync(h.inv_ell.p, inv.data(), sizeof(double) * h.d,
                              cudaMemcpyHostToDevice, h.stream));
    const int64_t tot = h.n * h.dp;
    prescale_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, h.stream>>>(
        h.X.p, h.n, h.d, h.dp, h.mu.p, h.inv_ell.p, std::sqrt(0.5), std::sqrt(0.5 * kLog2e),
        h.xs64.p, h.xs32.p);
    KPCG_LAUNCHED("prescale_kernel");
    KPCG_CUDA(cudaStreamSynchronize(h.stream));
}

static void check_theta(const double* log_theta, int n_theta, double noise) {
    if (!log_theta) fail(KPCG_ERR_ARG, "log_theta is NULL");
    for (int i = 0; i < n_theta; ++i)
        if (!std::isfinite(log_theta[i])) fail(KPCG_ERR_ARG, "log_theta has a non-finite entry");
    if (!(noise > 0.0) || !std::isfinite(noise)) fail(KPCG_ERR_ARG, "noise_var must be > 0");
}

void check_dev_ptr(const void* p, const char* name) {
    if (!p) fail(KPCG_ERR_ARG, std::string(name) + " is NULL");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(KPCG_ERR_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        fail(KPCG_ERR_ARG, std::string(name) + " is not a device pointer");
}

// ------------------------------------------------------------------ PCG
// Per-column batched PCG (Algorithm 1, textbook recurrence) in vector type T.
// X holds x0 on entry (zero if x0_zero) and the iterate on return.
// Returns the number of iterations run (max over columns).
// R0 (nullable, leading dimension h.ld) is the residual B - K_y X of the
// entry X when the caller has it, e.g. recomputed with a more accurate
// operator than `matvec`; then the recursion starts from it.
template <typename T, typename MV, typename PC>
static int pcg_core(Ctx& h, int c, const T* B, int64_t ldb, T* X, int64_t ldx, bool x0_zero,
                    double tol, int tol_mode, int max_iter, MV&& matvec, PC&& precond,
                    CgBufs<T>& bufs, std::vector<int>& iters_out, int& broken,
                    const T* R0 = nullptr) {
    const int64_t n = h.n, ld = h.ld;
    cudaStream_t st = h.stream;
    T* r = bufs.r.need((size_t)ld * c);
    T* z = bufs.z.need((size_t)ld * c);
    T* p = bufs.p.need((size_t)ld * c);
    T* q = bufs.q.need((size_t)ld * c);
    const int nblk = dot_blocks(n);
    double* partial = h.partial.need((size_t)nblk * c);
    double* sc = h.scal.need((size_t)6 * c);
    int* isc = h.iscal.need((size_t)2 * c + 2);
    CgScalars S{sc, sc + c, sc + 2 * c, sc + 3 * c, sc + 4 * c, sc + 5 * c, isc, isc + c,
                isc + 2 * c};
    KPCG_CUDA(cudaMemsetAsync(S.flags, 0, 2 * sizeof(int), st));
    ActiveScope active_scope(h, S.active);

    dot_cols<T>(B, ldb, B, ldb, n, c, partial, nblk, st);
    finalize(partial, nblk, c, FIN_NORM_B, S, tol, tol_mode, n, nullptr, st);
    if (x0_zero) {
        fill_zero_cols(X, sizeof(T), ldx, n, c, st);
        copy_cols<T>(r, ld, B, ldb, n, c, st);
    } else if (R0) {
        copy_cols<T>(r, ld, R0, ld, n, c, st);
    } else {
        matvec(X, ldx, c, q, ld);
        sub_cols_t_kernel<T><<<dim3(gx(n), c), 256, 0, st>>>(r, ld, B, ldb, q, ld, n);
        KPCG_LAUNCHED("sub_cols_t_kernel");
    }
    // initial stop test (no iteration counted)
    dot_cols<T>(r, ld, r, ld, n, c, partial, nblk, st);
    finalize(partial, nblk, c, FIN_RR, S, tol, tol_mode, n, nullptr, st);
    // FIN_RR counted one iteration for active columns: undo by resetting.
    KPCG_CUDA(cudaMemsetAsync(S.iters, 0, sizeof(int) * c, st));
    precond(r, ld, c, z, ld);
    copy_cols<T>(p, ld, z, ld, n, c, st);
    dot_cols<T>(r, ld, z, ld, n, c, partial, nblk, st);
    finalize(partial, nblk, c, FIN_RHO0, S, tol, tol_mode, n, nullptr, st);

    int it = 0;
    const int every = std::max(1, h.opt.check_every);
    int* hf = h.hflags;
    KPCG_CUDA(cudaMemcpyAsync(hf, S.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    int active = hf[0];
    // Graph path (h.use_graph, profiling off): after one plain chunk (which
    // makes every lazy allocation), `every` whole iterations and the read-back
    // of the activity flags are captured once into a CUDA graph and replayed.
    // Iterations past convergence inside a chunk change nothing: stopped
    // columns have alpha = beta = 0.
    GraphChunk chunk;
    const bool graphs = h.use_graph && !h.prof.on;
    auto body = [&](cudaStream_t s) {
        matvec(p, ld, c, q, ld);
        dot_cols<T>(p, ld, q, ld, n, c, partial, nblk, s);
        finalize(partial, nblk, c, FIN_ALPHA, S, tol, tol_mode, n, nullptr, s);
        update_xr<T>(X, ldx, r, ld, p, ld, q, ld, n, c, S.alpha, partial, nblk, s);
        finalize(partial, nblk, c, FIN_RR, S, tol, tol_mode, n, nullptr, s);
        precond(r, ld, c, z, ld);
        dot_cols<T>(r, ld, z, ld, n, c, partial, nblk, s);
        finalize(partial, nblk, c, FIN_BETA, S, tol, tol_mode, n, nullptr, s);
        update_p<T>(p, ld, z, ld, n, c, S.beta, S.active, s);
    };
    while (active > 0 && it < max_iter) {
        if (graphs && it >= every && it + every <= max_iter) {
            if (!chunk.exec)
                chunk.capture(h, [&](cudaStream_t cs) {
                    for (int j = 0; j < every; ++j) body(cs);
                    KPCG_CUDA(cudaMemcpyAsync(hf, S.flags, 2 * sizeof(int),
                                              cudaMemcpyDeviceToHost, cs));
                });
            KPCG_CUDA(cudaGraphLaunch(chunk.exec, st));
            note_launches(chunk.kernels);
            KPCG_CUDA(cudaStreamSynchronize(st));
            it += every;
            active = hf[0];
            continue;
        }
        matvec(p, ld, c, q, ld);
        dot_cols<T>(p, ld, q, ld, n, c, partial, nblk, st);
        finalize(partial, nblk, c, FIN_ALPHA, S, tol, tol_mode, n, nullptr, st);
        update_xr<T>(X, ldx, r, ld, p, ld, q, ld, n, c, S.alpha, partial, nblk, st);
        finalize(partial, nblk, c, FIN_RR, S, tol, tol_mode, n, nullptr, st);
        ++it;
        if (it % every == 0 || it >= max_iter) {
            KPCG_CUDA(cudaMemcpyAsync(hf, S.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            KPCG_CUDA(cudaStreamSynchronize(st));
            active = hf[0];
            if (active == 0) break;
        }
        precond(r, ld, c, z, ld);
        dot_cols<T>(r, ld, z, ld, n, c, partial, nblk, st);
        finalize(partial, nblk, c, FIN_BETA, S, tol, tol_mode, n, nullptr, st);
        update_p<T>(p, ld, z, ld, n, c, S.beta, S.active, st);
    }
    std::vector<int> its((size_t)c);
    KPCG_CUDA(cudaMemcpyAsync(its.data(), S.iters, sizeof(int) * c, cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaMemcpyAsync(hf, S.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    broken = hf[1];
    iters_out.assign(its.begin(), its.end());
    return it;
}

// Per-column ||B - K_y X||^2 and ||B||^2 in FP64 (host vectors).
static void residual_f64(Ctx& h, const double* B, int64_t ldb, int c, const double* X, int64_t ldx,
                         double* R, std::vector<double>& rr, std::vector<double>& bb,
                         bool double_float = false) {
    cudaStream_t st = h.stream;
    // symmetric tile pairs halve the FP64 exp work but take at most two
    // columns per pass; from three columns on, one non-symmetric pass over up
    // to 16 columns computes each entry's exp fewer times.  double_float: the
    // double-float product instead (a residual that only steers the iteration)
    h.prof.time(Profiler::RESID, st, [&] {
        if (double_float)
            kv_df(h, X, ldx, c, B, ldb, R, h.ld, h.noise);
        else if (c >= 3 && h.dp <= 16)
            kv_f64(h.xs64.p, h.n, h.dp, h.c0_64(), h.noise, X, ldx, c, B, ldb, R, h.ld, h.kvws,
                   st);
        else
            kv_f64_sym(h, X, ldx, c, B, ldb, R, h.ld, h.noise);
    });
    const int nblk = dot_blocks(h.n);
    double* partial = h.partial.need((size_t)nblk * c * 2);
    dot_cols<double>(R, h.ld, R, h.ld, h.n, c, partial, nblk, st);
    dot_cols<double>(B, ldb, B, ldb, h.n, c, partial + (size_t)nblk * c, nblk, st);
    std::vector<double> hp((size_t)nblk * c * 2);
    KPCG_CUDA(cudaMemcpyAsync(hp.data(), partial, sizeof(double) * hp.size(),
                              cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    rr.assign(c, 0.0);
    bb.assign(c, 0.0);
    for (int k = 0; k < c; ++k)
        for (int b = 0; b < nblk; ++b) {
            rr[k] += hp[(size_t)k * nblk + b];
            bb[k] += hp[(size_t)(c + k) * nblk + b];
        }
}

int pcg_f64(Ctx& h, int c, const double* B, int64_t ldb, double* X, int64_t ldx, bool x0_zero,
            double tol, int max_iter, const VecOp& matvec, const VecOp& precond,
            CgBufs<double>& bufs, std::vector<int>& iters, int& broken) {
    return pcg_core<double>(h, c, B, ldb, X, ldx, x0_zero, tol, 0, max_iter, matvec, precond,
                            bufs, iters, broken);
}

bool col_converged(double rr, double bb, double tol, int tol_mode, int64_t n) {
    if (bb == 0.0) return true;
    return tol_mode == 1 ? rr < (double)n * tol : rr <= tol * tol * bb;
}


// Noise of the system the preconditioner approximates: sigma^2 for the
// single-precision solvers, the shifted inner noise for the mixed ones.
static double precond_noise(const Ctx& h) {
    const bool mixed = h.opt.precision == KPCG_FP32_IR || h.opt.precision == KPCG_TC_IR ||
                       h.opt.precision == KPCG_FP32X_IR || h.opt.precision == KPCG_TCX_IR;
    return mixed ? h.noise * (1.0 + h.opt.inner_shift) : h.noise;
}

static void build_precond(Ctx& h) {
    h.P.reset();
    ++h.pversion;
    const double nz = precond_noise(h);
    if (h.pkind == KPCG_PREC_NYSTROM)
        nystrom_setup(h.P, h.xs32.p, h.xs64.p, h.n, h.dp, h.c0_32(), h.c0_64(), nz,
                      h.pidx.data(), h.psize, h.stream);
    else if (h.pkind == KPCG_PREC_BLOCK_JACOBI)
        block_jacobi_setup(h.P, h.xs64.p, h.n, h.dp, h.c0_64(), nz,
                           std::min<int64_t>(h.psize, h.n), h.stream);
    else if (h.pkind == KPCG_PREC_FITC)
        fitc_setup(h.P, h.xs32.p, h.xs64.p, h.n, h.dp, h.c0_32(), h.c0_64(), h.s2, nz,
                   h.pidx.data(), h.psize, h.stream);
    else if (h.pkind == KPCG_PREC_PITC)
        pitc_setup(h.P, h.xs32.p, h.xs64.p, h.n, h.dp, h.c0_64(), nz, h.pidx.data(), h.psize,
                   std::min<int64_t>(h.pblock, h.n), h.stream);
    else if (h.pkind == KPCG_PREC_SPECTRAL)
        spectral_setup(h.P, h.xs64.p, h.n, h.dp, h.s2, nz, h.pomega.data(), h.d, h.psize,
                       h.stream);
    h.P.n = h.n;
    h.P.noise = nz;
    KPCG_CUDA(cudaStreamSynchronize(h.stream));
}

// Rebuild the preconditioner if theta, the noise or the mode changed since.
double ensure_precond(Ctx& h) {
    h.P.n = h.n;
    if (h.pkind == KPCG_PREC_NONE) return 0.0;
    if (h.P.ready && h.P.noise == precond_noise(h)) return 0.0;
    const auto t0 = std::chrono::steady_clock::now();
    build_precond(h);
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Mixed precision.  Outer: flexible CG (Notay's FCG, the outer loop the
// paper uses around an inexact inner solve, Sec. 3.3.2) in FP64 with the
// FP64 operator; the A-orthogonalisation runs over a window of the last
// fcg_window directions.  Its preconditioner is an inner PCG in FP32 on the
// shifted operator K + sigma^2 (1 + shift) I, solved to inner_tol on the
// normalised residual.  The shift keeps the FP32 system positive definite
// when the FP32 rounding of K is not small against sigma^2; the outer loop
// removes the difference.  Columns are independent throughout.
kpcg_status fcg_solve(Ctx& h, const MixedOps& ops, const double* B, int64_t ldb, int c,
                      double tol, const double* X0, double* Xout, int64_t ldx,
                      std::vector<int>& iters_col, int& iters_total, int& steps,
                      std::vector<double>& rr, std::vector<double>& bb) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n, ld = h.ld;
    const int W = std::max(1, h.opt.fcg_window);
    double* R = h.R64.need((size_t)ld * c);
    double* Pw = h.fcgP.need((size_t)W * ld * c);
    double* APw = h.fcgAP.need((size_t)W * ld * c);
    double* Z = h.Q64.need((size_t)ld * c);
    float* b32 = h.c32.b.need((size_t)ld * c);
    float* d32 = h.c32.x.need((size_t)ld * c);
    double* cs = h.colscale.need((size_t)c * (W + 2));
    const int nblk = dot_blocks(n);
    double* partial = h.partial.need((size_t)nblk * c * (W + 2));
    std::vector<double> hp;
    auto dots = [&](int nd, const std::vector<std::pair<const double*, const double*>>& pairs,
                    std::vector<double>& out) {
        for (int t = 0; t < nd; ++t)
            dot_cols<double>(pairs[t].first, ld, pairs[t].second, ld, n, c,
                             partial + (size_t)t * nblk * c, nblk, st);
        hp.resize((size_t)nd * nblk * c);
        KPCG_CUDA(cudaMemcpyAsync(hp.data(), partial, sizeof(double) * hp.size(),
                                  cudaMemcpyDeviceToHost, st));
        KPCG_CUDA(cudaStreamSynchronize(st));
        out.assign((size_t)nd * c, 0.0);
        for (int t = 0; t < nd; ++t)
            for (int k = 0; k < c; ++k)
                for (int b2 = 0; b2 < nblk; ++b2)
                    out[(size_t)t * c + k] += hp[((size_t)t * c + k) * nblk + b2];
    };
    if (X0) {
        if (X0 != Xout) copy_cols<double>(Xout, ldx, X0, ldx, n, c, st);
        ops.residual(B, ldb, c, Xout, ldx, R, rr, bb, false);
    } else {
        // x0 = 0: the residual is B itself, no product needed
        fill_zero_cols(Xout, sizeof(double), ldx, n, c, st);
        copy_cols<double>(R, ld, B, ldb, n, c, st);
        dots(1, {{R, R}}, rr);
        bb = rr;
    }
    std::vector<double> pAp((size_t)W * c, 1.0), coef((size_t)c), d;
    std::vector<int> dead((size_t)c, 0);
    int nwin = 0, head = 0, stall = 0, recheck = 0;
    double best = INFINITY;
    kpcg_status status = KPCG_OK;
    for (int outer = 0;; ++outer) {
        bool all = true;
        double worst = 0.0;
        std::vector<double> scale((size_t)c, 0.0);
        for (int k = 0; k < c; ++k) {
            const bool ok = dead[k] || col_converged(rr[k], bb[k], tol, h.opt.tol_mode, n);
            all = all && ok;
            scale[k] = ok ? 0.0 : std::sqrt(rr[k]);
            if (bb[k] > 0 && !dead[k]) worst = std::max(worst, std::sqrt(rr[k] / bb[k]));
        }
        steps = outer;
        if (trace_on())
            std::fprintf(stderr, "kpcg fcg outer %d worst_rel_res %.3e inner_iters %d%s\n", outer,
                         worst, iters_total, recheck ? " (recomputed)" : "");
        if (all) {
            // certify on the recomputed residual; continue from it if the
            // recursive one drifted
            if (recheck) break;
            ops.residual(B, ldb, c, Xout, ldx, R, rr, bb, true);
            recheck = 1;
            nwin = 0;
            --outer;
            continue;
        }
        recheck = 0;
        if (outer >= h.opt.max_outer || iters_total >= h.opt.max_iter) {
            status = KPCG_ERR_NO_CONVERGENCE;
            break;
        }
        if (worst < best * 0.9) {
            best = worst;
            stall = 0;
        } else if (++stall >= 4) {
            status = KPCG_ERR_NO_CONVERGENCE;
            break;
        }
        // z = ||r|| * M(r / ||r||): inner PCG on the shifted operator, in FP32
        // vectors (or FP64 ones when the operator takes them)
        KPCG_CUDA(cudaMemcpyAsync(cs, scale.data(), sizeof(double) * c, cudaMemcpyHostToDevice,
                                  st));
        std::vector<int> its;
        int br = 0;
        const int budget = std::min(h.opt.inner_max_iter, h.opt.max_iter - iters_total);
        int ran;
        if (ops.inner_mv64) {
            double* b64 = h.c64.b.need((size_t)ld * c);
            double* d64 = h.c64.x.need((size_t)ld * c);
            convert_scale_cols<double, double>(b64, ld, R, ld, n, c, cs, 1, st);
            ran = pcg_core<double>(
                h, c, b64, ld, d64, ld, true, h.opt.inner_tol, 0, std::max(1, budget),
                [&](const double* V, int64_t ldv, int cc, double* O, int64_t ldo) {
                    h.prof.time(Profiler::KV_INNER, st,
                                [&] { ops.inner_mv64(V, ldv, cc, O, ldo); });
                },
                [&](const double* Rr, int64_t ldr, int cc, double* Zz, int64_t ldz) {
                    h.prof.time(Profiler::PRECOND, st,
                                [&] { ops.inner_pc64(Rr, ldr, cc, Zz, ldz); });
                },
                h.c64, its, br);
            convert_scale_cols<double, double>(Z, ld, d64, ld, n, c, cs, 0, st);
        } else {
            convert_scale_cols<float, double>(b32, ld, R, ld, n, c, cs, 1, st);
            ran = pcg_core<float>(
                h, c, b32, ld, d32, ld, true, h.opt.inner_tol, 0, std::max(1, budget),
                [&](const float* V, int64_t ldv, int cc, float* O, int64_t ldo) {
                    h.prof.time(Profiler::KV_INNER, st,
                                [&] { ops.inner_mv(V, ldv, cc, O, ldo); });
                },
                [&](const float* Rr, int64_t ldr, int cc, float* Zz, int64_t ldz) {
                    h.prof.time(Profiler::PRECOND, st,
                                [&] { ops.inner_pc(Rr, ldr, cc, Zz, ldz); });
                },
                h.c32, its, br);
            convert_scale_cols<double, float>(Z, ld, d32, ld, n, c, cs, 0, st);
        }
        iters_total += ran;
        // a bounded wait that expired inside the inner products ends the solve
        if (ops.timed_out && ops.timed_out())
            fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        for (int k = 0; k < c; ++k) iters_col[k] += (its[k] < 0 ? -1 - its[k] : its[k]);
        // p = z - sum_j (z^T A p_j / p_j^T A p_j) p_j over the window
        double* p = Pw + (size_t)head * ld * c;
        double* q = APw + (size_t)head * ld * c;
        if (nwin > 0) {
            std::vector<std::pair<const double*, const double*>> pr;
            std::vector<int> slot;
            for (int t = 0; t < nwin; ++t) {
                const int j = (head - 1 - t + W) % W;
                slot.push_back(j);
                pr.push_back({Z, APw + (size_t)j * ld * c});
            }
            dots(nwin, pr, d);
            std::vector<double> hc((size_t)nwin * c);
            for (int t = 0; t < nwin; ++t)
                for (int k = 0; k < c; ++k)
                    hc[(size_t)t * c + k] = -d[(size_t)t * c + k] / pAp[(size_t)slot[t] * c + k];
            KPCG_CUDA(cudaMemcpyAsync(cs + c, hc.data(), sizeof(double) * hc.size(),
                                      cudaMemcpyHostToDevice, st));
            copy_cols<double>(p, ld, Z, ld, n, c, st);
            for (int t = 0; t < nwin; ++t)
                axpy_cols_f64(p, ld, Pw + (size_t)slot[t] * ld * c, ld, n, c,
                              cs + c + (size_t)t * c, st);
        } else {
            copy_cols<double>(p, ld, Z, ld, n, c, st);
        }
        // columns that already meet tol have p = 0 exactly (zero right-hand side
        // for the inner solve, zero window coefficients); operators may skip them
        h.outer_cols.assign((size_t)c, 0);
        for (int k = 0; k < c; ++k) h.outer_cols[(size_t)k] = scale[k] > 0.0 ? 1 : 0;
        h.prof.time(Profiler::KV_OUTER, st, [&] { ops.outer_mv(p, ld, c, q, ld); });
        h.outer_cols.clear();
        dots(2, {{p, q}, {p, R}}, d);
        std::vector<double> al((size_t)c, 0.0), nal((size_t)c);
        for (int k = 0; k < c; ++k) {
            const double pq = d[k], pr = d[(size_t)c + k];
            pAp[(size_t)head * c + k] = (pq > 0.0) ? pq : 1.0;
            if (scale[k] > 0.0 && pq > 0.0 && std::isfinite(pq) && std::isfinite(pr))
                al[k] = pr / pq;
            else if (scale[k] > 0.0 && !(pq > 0.0))
                dead[k] = 1;  // breakdown of the outer recurrence for this column
            nal[k] = -al[k];
        }
        KPCG_CUDA(cudaMemcpyAsync(cs + c, al.data(), sizeof(double) * c, cudaMemcpyHostToDevice,
                                  st));
        KPCG_CUDA(cudaMemcpyAsync(cs + 2 * c, nal.data(), sizeof(double) * c,
                                  cudaMemcpyHostToDevice, st));
        axpy_cols_f64(Xout, ldx, p, ld, n, c, cs + c, st);
        axpy_cols_f64(R, ld, q, ld, n, c, cs + 2 * c, st);
        head = (head + 1) % W;
        nwin = std::min(nwin + 1, W);
        dots(1, {{R, R}}, rr);
    }
    for (int k = 0; k < c; ++k)
        if (dead[k] && status == KPCG_OK) status = KPCG_ERR_BREAKDOWN;
    if (ops.timed_out && ops.timed_out())
        fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
    return status;
}

// The operators of the single-problem mixed-precision solve.
static MixedOps single_ops(Ctx& h) {
    MixedOps o;
    const bool tc = (h.opt.precision == KPCG_TC_IR);
    const bool xf = (h.opt.precision == KPCG_FP32X_IR);
    const bool tcx = (h.opt.precision == KPCG_TCX_IR);
    const float inner_noise = (float)(h.noise * (1.0 + h.opt.inner_shift));
    Ctx* hp = &h;
    o.inner_mv = [hp, tc, xf, tcx, inner_noise](const float* V, int64_t ldv, int cc, float* O,
                                                int64_t ldo) {
        Ctx& h = *hp;
        if (tcx)
            kv_tcx_apply(h, V, ldv, cc, O, ldo, inner_noise);
        else if (tc)
            kv_tc_inner(h, V, ldv, cc, O, ldo, inner_noise);
        else if (xf)
            kv_xf(h, V, ldv, cc, O, ldo, inner_noise, 1);
        else
            kv_f32(h.xs32.p, h.n, h.dp, h.c0_32(), inner_noise, V, ldv, cc, O, ldo, h.kvws,
                   h.stream);
    };
    // Nystrom: the batched apply for one problem (one projection pass over up to
    // 16 columns, double-float back product); other kinds: the per-kind apply
    o.inner_pc = [hp](const float* R, int64_t ldr, int cc, float* Z, int64_t ldz) {
        Ctx& h = *hp;
        if ((h.P.kind == KPCG_PREC_NYSTROM || h.P.kind == KPCG_PREC_SPECTRAL) && h.P.ready) {
            if (h.nys1_c != cc || h.nys1_version != h.pversion) {
                nys_batch_plan(h.nys1, {&h.P}, cc, h.stream);
                h.nys1_c = cc;
                h.nys1_version = h.pversion;
            }
            nys_batch_apply(h.nys1, R, ldr, Z, ldz, h.n, nullptr, h.stream);
        } else {
            precond_apply_f32(h.P, R, ldr, cc, Z, ldz, h.stream);
        }
    };
    // directions of the outer loop: double-float (their product error scales
    // with the correction); true residuals stay native FP64 (residual_f64)
    o.outer_mv = [hp](const double* V, int64_t ldv, int cc, double* O, int64_t ldo) {
        kv_df(*hp, V, ldv, cc, nullptr, 0, O, ldo, hp->noise);
    };
    o.residual = [hp](const double* B, int64_t ldb, int cc, const double* X, int64_t ldx,
                      double* R, std::vector<double>& rr, std::vector<double>& bb, bool certify) {
        residual_f64(*hp, B, ldb, cc, X, ldx, R, rr, bb, !certify);
    };
    if (tc || tcx) o.timed_out = [hp]() { return kv_tc_error(*hp) != 0; };
    if (tcx && h.opt.inner_f64) {
        const double inner_noise64 = h.noise * (1.0 + h.opt.inner_shift);
        o.inner_mv64 = [hp, inner_noise64](const double* V, int64_t ldv, int cc, double* O,
                                           int64_t ldo) {
            kv_tcx_apply64(*hp, V, ldv, cc, O, ldo, inner_noise64);
        };
        // the preconditioner in FP32 between two conversions (its precision
        // does not decide the accuracy of the solve, only its speed)
        o.inner_pc64 = [hp, pc = o.inner_pc](const double* R, int64_t ldr, int cc, double* Z,
                                             int64_t ldz) {
            Ctx& h = *hp;
            float* r32 = h.c32.r.need((size_t)h.ld * cc);
            float* z32 = h.c32.z.need((size_t)h.ld * cc);
            convert_scale_cols<float, double>(r32, h.ld, R, ldr, h.n, cc, nullptr, 0, h.stream);
            pc(r32, h.ld, cc, z32, h.ld);
            convert_scale_cols<double, float>(Z, ldz, z32, h.ld, h.n, cc, nullptr, 0, h.stream);
        };
    }
    return o;
}

kpcg_status solve_impl(Ctx& h, const double* B, int64_t ldb, int c, double tol,
                              const double* X0, double* Xout, int64_t ldx, int32_t* iters_host,
                              kpcg_info* info) {
    const auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = launch_count();
    const double setup_ms = ensure_precond(h);
    h.prof.on = (h.opt.profile != 0);
    cudaStream_t st = h.stream;
    const int64_t n = h.n, ld = h.ld;
    const int prec = h.opt.precision;
    if (prec == KPCG_TC_IR && !kv_tc_supported(h.d))
        fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
    if (prec == KPCG_FP32X_IR && !kv_xf_supported(h))
        fail(KPCG_ERR_ARG, "exact-difference FP32 K.V needs d <= 16");
    if (prec == KPCG_TCX_IR && !kv_tcx_supported(h.d))
        fail(KPCG_ERR_ARG, "exact tensor-core K.V supports d <= 10");
    std::vector<int> iters_col((size_t)c, 0);
    int iters_total = 0, steps = 0, broken = 0;
    kpcg_status status = KPCG_OK;
    std::vector<double> rr, bb;
    bool rr_current = false;  // rr/bb hold the FP64 residual of the current Xout
    double* R = h.R64.need((size_t)ld * c);

    if (prec == KPCG_FP64 || prec == KPCG_FP32 || prec == KPCG_DF64) {
        // Plain PCG in one precision with residual replacement restarts.
        const bool f64 = (prec != KPCG_FP32);
        const bool dfk = (prec == KPCG_DF64);
        if (f64) {
            if (X0)
                copy_cols<double>(Xout, ldx, X0, ldx, n, c, st);
        }
        float* x32 = nullptr;
        float* b32 = nullptr;
        if (!f64) {
            x32 = h.c32.x.need((size_t)ld * c);
            b32 = h.c32.b.need((size_t)ld * c);
            convert_scale_cols<float, double>(b32, ld, B, ldb, n, c, nullptr, 0, st);
            if (X0) convert_scale_cols<float, double>(x32, ld, X0, ldx, n, c, nullptr, 0, st);
        }
        bool x0_zero = (X0 == nullptr);
        for (int pass = 0; pass <= std::max(0, h.opt.max_restarts); ++pass) {
            std::vector<int> its;
            int br = 0;
            const int budget = h.opt.max_iter - iters_total;
            if (budget <= 0) break;
            int ran;
            if (f64) {
                // The double-float operator differs from the FP64 one by ~1e-12
                // relative per entry; iterating to half the tolerance lets
                // the FP64 certification pass without a restart (a restart drops
                // the Krylov space and costs a second FP64 product).
                const double pass_tol = dfk ? 0.5 * tol : tol;
                ran = pcg_core<double>(
                    h, c, B, ldb, Xout, ldx, x0_zero, pass_tol, h.opt.tol_mode, budget,
                    [&](const double* V, int64_t ldv, int cc, double* O, int64_t ldo) {
                        h.prof.time(Profiler::KV_INNER, st, [&] {
                            if (dfk)
                                kv_df(h, V, ldv, cc, nullptr, 0, O, ldo, h.noise);
                            else if (cc >= 3 && h.dp <= 16)  // one pass over <= 16 columns
                                kv_f64(h.xs64.p, h.n, h.dp, h.c0_64(), h.noise, V, ldv, cc,
                                       nullptr, 0, O, ldo, h.kvws, h.stream);
                            else
                                kv_f64_sym(h, V, ldv, cc, nullptr, 0, O, ldo, h.noise);
                        });
                    },
                    [&](const double* Rr, int64_t ldr, int cc, double* Z, int64_t ldz) {
                        h.prof.time(Profiler::PRECOND, st, [&] {
                            precond_apply_f64(h.P, Rr, ldr, cc, Z, ldz, h.stream);
                        });
                    },
                    h.c64, its, br, rr_current ? R : nullptr);
            } else {
                ran = pcg_core<float>(
                    h, c, b32, ld, x32, ld, x0_zero, tol, h.opt.tol_mode, budget,
                    [&](const float* V, int64_t ldv, int cc, float* O, int64_t ldo) {
                        h.prof.time(Profiler::KV_INNER, st, [&] {
                            kv_f32(h.xs32.p, n, h.dp, h.c0_32(), (float)h.noise, V, ldv, cc, O,
                                   ldo, h.kvws, h.stream);
                        });
                    },
                    [&](const float* Rr, int64_t ldr, int cc, float* Z, int64_t ldz) {
                        h.prof.time(Profiler::PRECOND, st, [&] {
                            precond_apply_f32(h.P, Rr, ldr, cc, Z, ldz, h.stream);
                        });
                    },
                    h.c32, its, br);
            }
            iters_total += ran;
            for (int k = 0; k < c; ++k) iters_col[k] += std::abs(its[k] < 0 ? -1 - its[k] : its[k]);
            broken += br;
            x0_zero = false;
            rr_current = false;
            if (br) break;
            // true residual in the working precision decides a restart
            bool all = true;
            if (f64) {
                residual_f64(h, B, ldb, c, Xout, ldx, R, rr, bb);
                rr_current = true;
            } else {
                float* q32 = h.c32.q.need((size_t)ld * c);
                float* r32 = h.c32.r.need((size_t)ld * c);
                kv_f32(h.xs32.p, n, h.dp, h.c0_32(), (float)h.noise, x32, ld, c, q32, ld, h.kvws,
                       st);
                sub_cols_t_kernel<float><<<dim3(gx(n), c), 256, 0, st>>>(r32, ld, b32, ld, q32,
                                                                         ld, n);
                KPCG_LAUNCHED("sub_cols_t_kernel");
                const int nblk = dot_blocks(n);
                double* partial = h.partial.need((size_t)nblk * c * 2);
                dot_cols<float>(r32, ld, r32, ld, n, c, partial, nblk, st);
                dot_cols<float>(b32, ld, b32, ld, n, c, partial + (size_t)nblk * c, nblk, st);
                std::vector<double> hp((size_t)nblk * c * 2);
                KPCG_CUDA(cudaMemcpyAsync(hp.data(), partial, sizeof(double) * hp.size(),
                                          cudaMemcpyDeviceToHost, st));
                KPCG_CUDA(cudaStreamSynchronize(st));
                rr.assign(c, 0.0);
                bb.assign(c, 0.0);
                for (int k = 0; k < c; ++k)
                    for (int b = 0; b < nblk; ++b) {
                        rr[k] += hp[(size_t)k * nblk + b];
                        bb[k] += hp[(size_t)(c + k) * nblk + b];
                    }
            }
            for (int k = 0; k < c; ++k)
                all = all && col_converged(rr[k], bb[k], tol, h.opt.tol_mode, n);
            if (trace_on()) {
                double w = 0.0;
                for (int k = 0; k < c; ++k)
                    if (bb[k] > 0) w = std::max(w, std::sqrt(rr[k] / bb[k]));
                std::fprintf(stderr, "kpcg pass %d iters %d worst_rel_res %.3e%s\n", pass,
                             iters_total, w, br ? " (breakdown)" : "");
            }
            steps = pass;
            if (all || ran == 0) break;
        }
        if (!f64) convert_scale_cols<double, float>(Xout, ldx, x32, ld, n, c, nullptr, 0, st);
    } else {
        status = fcg_solve(h, single_ops(h), B, ldb, c, tol, X0, Xout, ldx, iters_col, iters_total,
                           steps, rr, bb);
        rr_current = (status == KPCG_OK);  // converged exits certify on a recomputed residual
    }
    // FP64 residual of what is returned (the single-precision FP32 solver
    // checked its own operator only)
    double maxrel = 0.0;
    if (!rr_current || prec == KPCG_FP32) residual_f64(h, B, ldb, c, Xout, ldx, R, rr, bb);
    bool all = true;
    for (int k = 0; k < c; ++k) {
        if (bb[k] > 0) maxrel = std::max(maxrel, std::sqrt(rr[k] / bb[k]));
        all = all && col_converged(rr[k], bb[k], tol, h.opt.tol_mode, n);
    }
    if (status == KPCG_OK && !all) status = broken ? KPCG_ERR_BREAKDOWN : KPCG_ERR_NO_CONVERGENCE;
    if (iters_host)
        for (int k = 0; k < c; ++k) iters_host[k] = iters_col[k];
    if (info) {
        info->iters_total = iters_total;
        info->outer_steps = steps;
        info->max_rel_res = maxrel;
        info->time_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
        info->setup_ms = setup_ms;
        double ms[Profiler::NCAT];
        int calls[Profiler::NCAT];
        KPCG_CUDA(cudaStreamSynchronize(st));
        h.prof.collect(ms, calls);
        info->kv_inner_ms = ms[Profiler::KV_INNER];
        info->kv_inner_calls = calls[Profiler::KV_INNER];
        info->kv_outer_ms = ms[Profiler::KV_OUTER];
        info->kv_outer_calls = calls[Profiler::KV_OUTER];
        info->precond_ms = ms[Profiler::PRECOND];
        info->precond_calls = calls[Profiler::PRECOND];
        info->resid_ms = ms[Profiler::RESID];
        info->resid_calls = calls[Profiler::RESID];
        info->launches = (int)(launch_count() - launches0);
        info->precond_jitter = h.P.ready ? h.P.jitter : 0.0;
    } else {
        double ms[Profiler::NCAT];
        int calls[Profiler::NCAT];
        KPCG_CUDA(cudaStreamSynchronize(st));
        h.prof.collect(ms, calls);
    }
    if (status != KPCG_OK)
        h.err = std::string(kpcg_status_string(status)) +
                ": max relative residual " + std::to_string(maxrel);
    return status;
}

// Slot of the j-th most recent snapshot (j = 0: newest).
static int snap_slot(const Ctx& h, int j) { return ((h.whead - 1 - j) % h.wq + h.wq) % h.wq; }

__global__ void snap_expand_kernel(const double* __restrict__ S, int64_t ld, int q, int head,
                                   int count, const double* __restrict__ c,
                                   double* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < count; ++j) {
            const int slot = ((head - 1 - j) % q + q) % q;
            s = fma(c[j], S[(int64_t)slot * ld + i], s);
        }
        x[i] = s;
    }
}

// c = argmin |S c - a|^2 + ridge (tr(G)/q) |c|^2 over the stored snapshots:
// G = S^T S and S^T a by the FP64 dot kernels, then a q x q Cholesky solve
// (at most 16 unknowns) on the host; coefficients of missing snapshots are 0.
void snapshot_fit(Ctx& h, const double* a, double* c_dev) {
    cudaStream_t st = h.stream;
    const int q = h.wq, cnt = h.wcount;
    std::vector<double> c((size_t)q, 0.0);
    if (cnt > 0) {
        const int nblk = dot_blocks(h.n);
        const int npair = cnt * (cnt + 1) / 2 + cnt;
        double* partial = h.partial.need((size_t)nblk * npair);
        int t = 0;
        for (int i = 0; i < cnt; ++i) {
            const double* Si = h.wsnap.p + (size_t)snap_slot(h, i) * h.ld;
            for (int j = 0; j <= i; ++j, ++t)
                dot_cols<double>(Si, h.ld, h.wsnap.p + (size_t)snap_slot(h, j) * h.ld, h.ld, h.n,
                                 1, partial + (size_t)t * nblk, nblk, st);
            dot_cols<double>(Si, h.ld, a, h.ld, h.n, 1,
                             partial + (size_t)(cnt * (cnt + 1) / 2 + i) * nblk, nblk, st);
        }
        std::vector<double> hp((size_t)nblk * npair);
        KPCG_CUDA(cudaMemcpyAsync(hp.data(), partial, sizeof(double) * hp.size(),
                                  cudaMemcpyDeviceToHost, st));
        KPCG_CUDA(cudaStreamSynchronize(st));
        auto sum = [&](int idx) {
            double v = 0.0;
            for (int b = 0; b < nblk; ++b) v += hp[(size_t)idx * nblk + b];
            return v;
        };
        std::vector<double> G((size_t)cnt * cnt), r((size_t)cnt);
        t = 0;
        for (int i = 0; i < cnt; ++i)
            for (int j = 0; j <= i; ++j, ++t) G[(size_t)i * cnt + j] = G[(size_t)j * cnt + i] = sum(t);
        double tr = 0.0;
        for (int i = 0; i < cnt; ++i) {
            r[(size_t)i] = sum(cnt * (cnt + 1) / 2 + i);
            tr += G[(size_t)i * cnt + i];
        }
        for (int i = 0; i < cnt; ++i) G[(size_t)i * cnt + i] += h.wridge * tr / cnt;
        // Cholesky G = L L^T in place (lower), then two triangular solves
        for (int j = 0; j < cnt; ++j) {
            double d = G[(size_t)j * cnt + j];
            for (int k = 0; k < j; ++k) d -= G[(size_t)j * cnt + k] * G[(size_t)j * cnt + k];
            if (!(d > 0.0)) fail(KPCG_ERR_NOT_SPD, "snapshot Gram matrix not positive definite");
            d = std::sqrt(d);
            G[(size_t)j * cnt + j] = d;
            for (int i = j + 1; i < cnt; ++i) {
                double v = G[(size_t)i * cnt + j];
                for (int k = 0; k < j; ++k) v -= G[(size_t)i * cnt + k] * G[(size_t)j * cnt + k];
                G[(size_t)i * cnt + j] = v / d;
            }
        }
        for (int i = 0; i < cnt; ++i) {
            double v = r[(size_t)i];
            for (int k = 0; k < i; ++k) v -= G[(size_t)i * cnt + k] * c[(size_t)k];
            c[(size_t)i] = v / G[(size_t)i * cnt + i];
        }
        for (int i = cnt - 1; i >= 0; --i) {
            double v = c[(size_t)i];
            for (int k = i + 1; k < cnt; ++k) v -= G[(size_t)k * cnt + i] * c[(size_t)k];
            c[(size_t)i] = v / G[(size_t)i * cnt + i];
        }
    }
    KPCG_CUDA(cudaMemcpyAsync(c_dev, c.data(), sizeof(double) * q, cudaMemcpyHostToDevice, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
}

void snapshot_expand(Ctx& h, const double* c, double* x0) {
    const int blocks = (int)std::min<int64_t>((h.n + 255) / 256, 152 * 8);
    snap_expand_kernel<<<blocks, 256, 0, h.stream>>>(h.wsnap.p, h.ld, h.wq, h.whead, h.wcount, c,
                                                      x0, h.n);
    KPCG_LAUNCHED("snap_expand_kernel");
    KPCG_CUDA(cudaStreamSynchronize(h.stream));
}

}  // namespace kpcg

using kpcg::Ctx;
using kpcg::fail;


#define KPCG_GUARD(hptr, ...)                                               \
    try {                                                                   \
        __VA_ARGS__;                                                        \
    } catch (const kpcg::Error& e) {                                        \
        if (hptr) (hptr)->err = e.msg;                                      \
        else kpcg::g_create_err = e.msg;                                    \
        return e.status;                                                    \
    } catch (const std::exception& e) {                                     \
        if (hptr) (hptr)->err = e.what();                                   \
        else kpcg::g_create_err = e.what();                                 \
        return KPCG_ERR_ARG;                                                \
    }

extern "C" {

void kpcg_default_options(kpcg_options* opt) {
    if (!opt) return;
    opt->max_iter = 100000;
    opt->precision = KPCG_FP32_IR;
    opt->tol_mode = 0;
    opt->max_outer = 60;
    opt->inner_tol = 1e-2;
    opt->check_every = 4;
    opt->max_restarts = 5;
    opt->inner_shift = 1.0;
    opt->inner_max_iter = 2000;
    opt->fcg_window = 16;
    opt->profile = 0;
    opt->wait_stall = 0;
    opt->wait_limit_ns = 0;
    opt->inner_f64 = 0;
}

const char* kpcg_status_string(kpcg_status s) {
    switch (s) {
        case KPCG_OK: return "KPCG_OK";
        case KPCG_ERR_ARG: return "KPCG_ERR_ARG";
        case KPCG_ERR_CUDA: return "KPCG_ERR_CUDA";
        case KPCG_ERR_OOM: return "KPCG_ERR_OOM";
        case KPCG_ERR_NOT_SPD: return "KPCG_ERR_NOT_SPD";
        case KPCG_ERR_BREAKDOWN: return "KPCG_ERR_BREAKDOWN";
        case KPCG_ERR_NO_CONVERGENCE: return "KPCG_ERR_NO_CONVERGENCE";
        case KPCG_ERR_TIMEOUT: return "KPCG_ERR_TIMEOUT";
        case KPCG_ERR_STATE: return "KPCG_ERR_STATE";
    }
    return "KPCG_UNKNOWN";
}

static void check_opts(const kpcg_options* o) {
    if (o->max_iter < 0 || o->max_outer < 0 || o->check_every < 1 || o->max_restarts < 0)
        fail(KPCG_ERR_ARG, "invalid options");
    if (o->precision < KPCG_FP64 || o->precision > KPCG_TCX_IR)
        fail(KPCG_ERR_ARG, "invalid precision");
    if (o->tol_mode != 0 && o->tol_mode != 1) fail(KPCG_ERR_ARG, "invalid tol_mode");
    if (!(o->inner_tol > 0.0 && o->inner_tol < 1.0)) fail(KPCG_ERR_ARG, "inner_tol not in (0,1)");
    if (!(o->inner_shift >= 0.0) || !std::isfinite(o->inner_shift))
        fail(KPCG_ERR_ARG, "inner_shift must be >= 0");
    if (o->inner_max_iter < 1 || o->fcg_window < 1 || o->fcg_window > 64)
        fail(KPCG_ERR_ARG, "inner_max_iter >= 1 and fcg_window in [1, 64] required");
    if (o->wait_stall != 0 && o->wait_stall != 1) fail(KPCG_ERR_ARG, "wait_stall must be 0 or 1");
    if (o->inner_f64 != 0 && o->inner_f64 != 1) fail(KPCG_ERR_ARG, "inner_f64 must be 0 or 1");
    if (o->wait_limit_ns < 0 || o->wait_limit_ns > (int64_t)60000000000)
        fail(KPCG_ERR_ARG, "wait_limit_ns must be in [0, 60 s]");
}

kpcg_status kpcg_create(const float* X, int64_t n, int32_t d, const double* log_theta, int32_t ard,
                        double noise_var, const kpcg_options* opt, void* stream, kpcg_t* out) {
    kpcg_ctx* h = nullptr;
    try {
        if (!out) fail(KPCG_ERR_ARG, "out is NULL");
        *out = nullptr;
        if (n < 1) fail(KPCG_ERR_ARG, "n must be >= 1");
        if (n > (int64_t)1 << 31) fail(KPCG_ERR_ARG, "n too large");
        if (d < 1 || kpcg::padded_dim(d) < 0) fail(KPCG_ERR_ARG, "d must be in [1, 32]");
        kpcg::check_theta(log_theta, ard ? d + 1 : 2, noise_var);
        kpcg::check_dev_ptr(X, "X");
        if (((uintptr_t)X) % 4) fail(KPCG_ERR_ARG, "X must be 4-byte aligned");
        h = new kpcg_ctx();
        h->use_graph = true;  // replay CG chunks from graphs whenever profiling is off
        KPCG_CUDA(cudaGetDevice(&h->device));
        h->stream = (cudaStream_t)stream;
        h->n = n;
        h->ld = ((n + 31) / 32) * 32;
        h->d = d;
        h->dp = kpcg::padded_dim(d);
        h->ard = ard ? 1 : 0;
        h->log_theta.assign(log_theta, log_theta + (ard ? d + 1 : 2));
        h->noise = noise_var;
        kpcg_default_options(&h->opt);
        if (opt) {
            check_opts(opt);
            h->opt = *opt;
        }
        KPCG_CUDA(cudaHostAlloc((void**)&h->hflags, 4 * sizeof(int), cudaHostAllocDefault));
        h->X.need((size_t)n * d);
        KPCG_CUDA(cudaMemcpyAsync(h->X.p, X, sizeof(float) * n * d, cudaMemcpyDeviceToDevice,
                                  h->stream));
        h->mu.need(d);
        h->inv_ell.need(d);
        h->xs64.need((size_t)n * h->dp);
        h->xs32.need((size_t)n * h->dp);
        kpcg::colmean_kernel<<<d, 256, 0, h->stream>>>(h->X.p, n, d, h->mu.p);
        KPCG_LAUNCHED("colmean_kernel");
        kpcg::ctx_rescale(*h);
        *out = h;
        return KPCG_OK;
    } catch (const kpcg::Error& e) {
        kpcg::g_create_err = e.msg;
        if (h) {
            if (h->hflags) cudaFreeHost(h->hflags);
            delete h;
        }
        return e.status;
    }
}

kpcg_status kpcg_set_theta(kpcg_t h, const double* log_theta, double noise_var) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        kpcg::check_theta(log_theta, h->ard ? h->d + 1 : 2, noise_var);
        h->log_theta.assign(log_theta, log_theta + (h->ard ? h->d + 1 : 2));
        h->noise = noise_var;
        h->P.reset();
        h->Wb.reset();
        kpcg::ctx_rescale(*h);
    });
    return KPCG_OK;
}

kpcg_status kpcg_set_options(kpcg_t h, const kpcg_options* opt) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (!opt) fail(KPCG_ERR_ARG, "opt is NULL");
        check_opts(opt);
        h->opt = *opt;
    });
    return KPCG_OK;
}

kpcg_status kpcg_precond(kpcg_t h, int32_t kind, int64_t size, const int64_t* idx) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (kind == KPCG_PREC_NYSTROM || kind == KPCG_PREC_FITC) {
            if (size < 1 || size > h->n || size > 4096)
                fail(KPCG_ERR_ARG, "inducing-point count m must be in [1, min(n, 4096)]");
            if (!idx) fail(KPCG_ERR_ARG, "Nystrom and FITC need the inducing indices");
            for (int64_t a = 0; a < size; ++a) {
                if (idx[a] < 0 || idx[a] >= h->n) fail(KPCG_ERR_ARG, "inducing index out of range");
                if (a && idx[a] <= idx[a - 1])
                    fail(KPCG_ERR_ARG, "inducing indices must be sorted and distinct");
            }
            h->pidx.assign(idx, idx + size);
        } else if (kind == KPCG_PREC_BLOCK_JACOBI) {
            if (size < 1 || size > 4096) fail(KPCG_ERR_ARG, "block size must be in [1, 4096]");
            h->pidx.clear();
        } else if (kind == KPCG_PREC_NONE) {
            h->pidx.clear();
        } else if (kind == KPCG_PREC_SPECTRAL) {
            fail(KPCG_ERR_ARG, "the random-feature preconditioner is built by kpcg_precond_spectral");
        } else if (kind == KPCG_PREC_PITC) {
            fail(KPCG_ERR_ARG, "PITC is built by kpcg_precond_pitc");
        } else {
            fail(KPCG_ERR_ARG, "unknown preconditioner kind");
        }
        h->pkind = KPCG_PREC_NONE;
        h->P.reset();
        h->pkind = kind;
        h->psize = size;
        if (kind != KPCG_PREC_NONE) {
            try {
                kpcg::build_precond(*h);
            } catch (...) {
                h->pkind = KPCG_PREC_NONE;
                h->P.reset();
                throw;
            }
        }
    });
    return KPCG_OK;
}

kpcg_status kpcg_precond_pitc(kpcg_t h, int64_t m, const int64_t* idx, int64_t b) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (m < 1 || m > h->n || m > 4096)
            fail(KPCG_ERR_ARG, "inducing-point count m must be in [1, min(n, 4096)]");
        if (b < 1 || b > 4096) fail(KPCG_ERR_ARG, "block size must be in [1, 4096]");
        if (!idx) fail(KPCG_ERR_ARG, "PITC needs the inducing indices");
        for (int64_t a = 0; a < m; ++a) {
            if (idx[a] < 0 || idx[a] >= h->n) fail(KPCG_ERR_ARG, "inducing index out of range");
            if (a && idx[a] <= idx[a - 1])
                fail(KPCG_ERR_ARG, "inducing indices must be sorted and distinct");
        }
        h->pkind = KPCG_PREC_NONE;
        h->P.reset();
        h->pidx.assign(idx, idx + m);
        h->pkind = KPCG_PREC_PITC;
        h->psize = m;
        h->pblock = b;
        try {
            kpcg::build_precond(*h);
        } catch (...) {
            h->pkind = KPCG_PREC_NONE;
            h->P.reset();
            throw;
        }
    });
    return KPCG_OK;
}

kpcg_status kpcg_precond_spectral(kpcg_t h, int64_t m, const double* omega) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (m < 1 || m > 2048) fail(KPCG_ERR_ARG, "feature count m must be in [1, 2048]");
        if (!omega) fail(KPCG_ERR_ARG, "omega (host, m x d) is required");
        const size_t cnt = (size_t)m * (size_t)h->d;
        for (size_t e = 0; e < cnt; ++e)
            if (!std::isfinite(omega[e])) fail(KPCG_ERR_ARG, "omega has a non-finite value");
        h->pkind = KPCG_PREC_NONE;
        h->P.reset();
        h->pidx.clear();
        h->pomega.assign(omega, omega + cnt);
        h->pkind = KPCG_PREC_SPECTRAL;
        h->psize = m;
        try {
            kpcg::build_precond(*h);
        } catch (...) {
            h->pkind = KPCG_PREC_NONE;
            h->P.reset();
            throw;
        }
    });
    return KPCG_OK;
}

kpcg_status kpcg_matvec_f64(kpcg_t h, const double* V, int64_t ldv, int32_t c, double* O,
                            int64_t ldo, int32_t impl) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (c < 0 || ldv < h->n || ldo < h->n) fail(KPCG_ERR_ARG, "bad sizes");
        if (c == 0) return KPCG_OK;
        kpcg::check_dev_ptr(V, "V");
        kpcg::check_dev_ptr(O, "O");
        if (impl == 0)
            kpcg::kv_f64_sym(*h, V, ldv, c, nullptr, 0, O, ldo, h->noise);
        else if (impl == 1) {
            kpcg::kv_df(*h, V, ldv, c, nullptr, 0, O, ldo, h->noise);
            if (kpcg::kv_tc_error(*h))
                fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        } else if (impl == 3) {
            // the double-float kernel on the FP32 pipe alone (no tensor-core distances)
            const bool saved = h->df_tensor;
            h->df_tensor = false;
            try {
                kpcg::kv_df(*h, V, ldv, c, nullptr, 0, O, ldo, h->noise);
            } catch (...) {
                h->df_tensor = saved;
                throw;
            }
            h->df_tensor = saved;
        } else if (impl == 4) {
            // the tensor-core double-float product evaluating every entry
            if (!kpcg::kv_tcd_supported(*h))
                fail(KPCG_ERR_ARG, "the double-float tensor-core K.V needs d <= 10");
            const bool saved = h->tcd_symmetric;
            h->tcd_symmetric = false;
            try {
                kpcg::kv_tcd(*h, V, ldv, c, nullptr, 0, O, ldo, h->noise);
            } catch (...) {
                h->tcd_symmetric = saved;
                throw;
            }
            h->tcd_symmetric = saved;
            if (kpcg::kv_tc_error(*h))
                fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        } else if (impl == 2) {
            if (!kpcg::kv_tcx_supported(h->d))
                fail(KPCG_ERR_ARG, "exact tensor-core K.V supports d <= 10");
            kpcg::kv_tcx_apply64(*h, V, ldv, c, O, ldo, h->noise);
            if (kpcg::kv_tc_error(*h))
                fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        } else
            fail(KPCG_ERR_ARG, "unknown impl");
        KPCG_CUDA(cudaStreamSynchronize(h->stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_matvec_f32(kpcg_t h, const float* V, int64_t ldv, int32_t c, float* O,
                            int64_t ldo, int32_t impl) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (c < 0 || ldv < h->n || ldo < h->n) fail(KPCG_ERR_ARG, "bad sizes");
        if (c == 0) return KPCG_OK;
        kpcg::check_dev_ptr(V, "V");
        kpcg::check_dev_ptr(O, "O");
        if (impl == 0) {
            kpcg::kv_f32(h->xs32.p, h->n, h->dp, h->c0_32(), (float)h->noise, V, ldv, c, O, ldo,
                         h->kvws, h->stream);
        } else if (impl == 1) {
            if (!kpcg::kv_tc_supported(h->d))
                fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
            kpcg::kv_tc_apply(*h, V, ldv, c, O, ldo, (float)h->noise);
            if (kpcg::kv_tc_error(*h))
                fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        } else if (impl == 2 || impl == 3) {
            if (!kpcg::kv_xf_supported(*h))
                fail(KPCG_ERR_ARG, "exact-difference FP32 K.V needs d <= 16");
            kpcg::kv_xf(*h, V, ldv, c, O, ldo, (float)h->noise, impl - 2);
        } else if (impl == 4) {
            if (!kpcg::kv_tcx_supported(h->d))
                fail(KPCG_ERR_ARG, "exact tensor-core K.V supports d <= 10");
            kpcg::kv_tcx_apply(*h, V, ldv, c, O, ldo, (float)h->noise);
            if (kpcg::kv_tc_error(*h))
                fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        } else if (impl == 5) {
            if (!kpcg::kv_tcv_supported(h->d))
                fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
            kpcg::kv_tcv_apply(*h, V, ldv, c, O, ldo, (float)h->noise);
            if (kpcg::kv_tc_error(*h))
                fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        } else if (impl == 6) {
            if (!kpcg::kv_tc_supported(h->d))
                fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
            if (kpcg::kv_tcs_usable(*h))
                kpcg::kv_tcs_apply(*h, V, ldv, c, O, ldo, (float)h->noise);
            else  // a single tile has no symmetric pairs
                kpcg::kv_tc_apply(*h, V, ldv, c, O, ldo, (float)h->noise);
            if (kpcg::kv_tc_error(*h))
                fail(KPCG_ERR_TIMEOUT, "a bounded wait in the tensor-core K.V expired");
        } else {
            fail(KPCG_ERR_ARG, "unknown impl");
        }
        KPCG_CUDA(cudaStreamSynchronize(h->stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_precond_apply_f64(kpcg_t h, const double* R, int64_t ldr, int32_t c, double* Z,
                                   int64_t ldz) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (c < 0 || ldr < h->n || ldz < h->n) fail(KPCG_ERR_ARG, "bad sizes");
        if (c == 0) return KPCG_OK;
        kpcg::check_dev_ptr(R, "R");
        kpcg::check_dev_ptr(Z, "Z");
        kpcg::ensure_precond(*h);
        kpcg::precond_apply_f64(h->P, R, ldr, c, Z, ldz, h->stream);
        KPCG_CUDA(cudaStreamSynchronize(h->stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_solve(kpcg_t h, const double* B, int64_t ldb, int32_t c, double tol,
                       const double* X0, double* Xout, int64_t ldx, int32_t* iters,
                       kpcg_info* info) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (c < 0 || ldb < h->n || ldx < h->n) fail(KPCG_ERR_ARG, "bad sizes");
        if (!(tol > 0.0)) fail(KPCG_ERR_ARG, "tol must be > 0");
        if (c == 0) return KPCG_OK;
        kpcg::check_dev_ptr(B, "B");
        kpcg::check_dev_ptr(Xout, "Xout");
        if (X0) kpcg::check_dev_ptr(X0, "X0");
        h->P.n = h->n;
        return kpcg::solve_impl(*h, B, ldb, c, tol, X0, Xout, ldx, iters, info);
    });
    return KPCG_OK;
}

kpcg_status kpcg_dkv(kpcg_t h, const double* W, int64_t ldw, int32_t c, double* G, int64_t ldg) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (c < 0 || ldw < h->n || ldg < h->n) fail(KPCG_ERR_ARG, "bad sizes");
        if (c == 0) return KPCG_OK;
        kpcg::check_dev_ptr(W, "W");
        kpcg::check_dev_ptr(G, "G");
        kpcg::dkv_f64(h->xs64.p, h->n, h->dp, h->d, h->ard, h->c0_64(), W, ldw, c, G, ldg,
                      h->kvws, h->stream);
        KPCG_CUDA(cudaStreamSynchronize(h->stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_grad(kpcg_t h, const double* y, const double* probes, int32_t t, double tol,
                      const double* alpha0, double* grad, double* alpha, kpcg_info* info) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (t < 1) fail(KPCG_ERR_ARG, "t must be >= 1");
        if (!grad) fail(KPCG_ERR_ARG, "grad is NULL");
        kpcg::check_dev_ptr(y, "y");
        kpcg::check_dev_ptr(probes, "probes");
        if (alpha) kpcg::check_dev_ptr(alpha, "alpha");
        const int64_t n = h->n, ld = h->ld;
        const int c = t + 1;
        cudaStream_t st = h->stream;
        double* Bb = h->Bblk.need((size_t)ld * c);
        double* Sb = h->Sblk.need((size_t)ld * c);
        kpcg::copy_cols<double>(Bb, ld, y, n, n, 1, st);
        kpcg::copy_cols<double>(Bb + ld, ld, probes, n, n, t, st);
        kpcg_info sinfo{};
        h->P.n = n;
        const double* X0 = nullptr;
        if (alpha0) {
            kpcg::check_dev_ptr(alpha0, "alpha0");
            double* X0b = h->Q64.need((size_t)ld * c);
            kpcg::fill_zero_cols(X0b, sizeof(double), ld, n, c, st);
            kpcg::copy_cols<double>(X0b, ld, alpha0, n, n, 1, st);
            X0 = X0b;
        }
        const kpcg_status s = kpcg::solve_impl(*h, Bb, ld, c, tol, X0, Sb, ld, nullptr, &sinfo);
        if (s != KPCG_OK) return s;
        // G_q = dK_q [a, r_1..r_t]
        const int nq = (h->ard ? h->d : 1) + 1;
        double* W64 = h->Q64.need((size_t)ld * c);
        kpcg::copy_cols<double>(W64, ld, Sb, ld, n, 1, st);
        kpcg::copy_cols<double>(W64 + ld, ld, probes, n, n, t, st);
        double* G = h->G.need((size_t)nq * ld * c);
        // double-float entries and sums (the trace term cancels all but ~1e-5
        // of the magnitude of dK W); native FP64 above d = 16
        if (h->dp <= 16)
            kpcg::dkv_df(*h, W64, ld, c, G, ld);
        else
            kpcg::dkv_f64(h->xs64.p, n, h->dp, h->d, h->ard, h->c0_64(), W64, ld, c, G, ld,
                          h->kvws, st);
        // dots: S^T G_q per column (c of them), and S^T [a, r_1..r_t] for the noise term
        kpcg::copy_cols<double>(Bb, ld, Sb, ld, n, 1, st);
        const int nblk = kpcg::dot_blocks(n);
        double* partial = h->partial.need((size_t)nblk * c * (nq + 1));
        for (int q = 0; q < nq; ++q)
            kpcg::dot_cols<double>(Sb, ld, G + (size_t)q * ld * c, ld, n, c,
                                   partial + (size_t)q * nblk * c, nblk, st);
        kpcg::dot_cols<double>(Sb, ld, Bb, ld, n, c, partial + (size_t)nq * nblk * c, nblk, st);
        std::vector<double> hp((size_t)nblk * c * (nq + 1));
        KPCG_CUDA(cudaMemcpyAsync(hp.data(), partial, sizeof(double) * hp.size(),
                                  cudaMemcpyDeviceToHost, st));
        if (alpha) kpcg::copy_cols<double>(alpha, n, Sb, ld, n, 1, st);
        KPCG_CUDA(cudaStreamSynchronize(st));
        auto dot = [&](int q, int k) {
            double s = 0.0;
            for (int b = 0; b < nblk; ++b) s += hp[((size_t)q * c + k) * nblk + b];
            return s;
        };
        for (int q = 0; q <= nq; ++q) {
            double tr = 0.0;
            for (int k = 1; k < c; ++k) tr += dot(q, k);
            tr /= (double)t;
            const double quad = dot(q, 0);
            const double scale = (q == nq) ? h->noise : 1.0;  // dK_y/dlog sigma^2 = sigma^2 I
            grad[q] = scale * (-0.5 * tr + 0.5 * quad);
        }
        if (info) *info = sinfo;
    });
    return KPCG_OK;
}

kpcg_status kpcg_warm_basis(kpcg_t h, int64_t m, const int64_t* idx, double ridge) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (m < 1 || m > h->n || m > 4096) fail(KPCG_ERR_ARG, "m must be in [1, min(n, 4096)]");
        if (!idx) fail(KPCG_ERR_ARG, "idx is NULL");
        if (!(ridge > 0.0) || !std::isfinite(ridge)) fail(KPCG_ERR_ARG, "ridge must be > 0");
        for (int64_t a = 0; a < m; ++a) {
            if (idx[a] < 0 || idx[a] >= h->n) fail(KPCG_ERR_ARG, "basis index out of range");
            if (a && idx[a] <= idx[a - 1]) fail(KPCG_ERR_ARG, "basis indices must be sorted");
        }
        h->widx.assign(idx, idx + m);
        h->wridge = ridge;
        h->Wb.reset();
        h->wmode = 1;
    });
    return KPCG_OK;
}

static void ensure_warm(kpcg::Ctx& h) {
    if (h.wmode != 1 || h.widx.empty())
        fail(KPCG_ERR_STATE, "no warm-start basis: call kpcg_warm_basis first");
    if (h.Wb.ready) return;
    kpcg::nystrom_setup(h.Wb, h.xs32.p, h.xs64.p, h.n, h.dp, h.c0_32(), h.c0_64(), h.wridge,
                        h.widx.data(), (int64_t)h.widx.size(), h.stream);
    h.Wb.n = h.n;
}

kpcg_status kpcg_warm_snapshots(kpcg_t h, int32_t q, double ridge) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (q < 1 || q > 16) fail(KPCG_ERR_ARG, "q must be in [1, 16]");
        if (!(ridge > 0.0) || !std::isfinite(ridge)) fail(KPCG_ERR_ARG, "ridge must be > 0");
        h->wsnap.need((size_t)q * h->ld);
        h->wc.need(16);
        h->wq = q;
        h->wcount = 0;
        h->whead = 0;
        h->wridge = ridge;
        h->wmode = 2;
    });
    return KPCG_OK;
}

kpcg_status kpcg_warm_push(kpcg_t h, const double* a) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        if (h->wmode != 2) fail(KPCG_ERR_STATE, "no snapshot basis: call kpcg_warm_snapshots first");
        kpcg::check_dev_ptr(a, "a");
        KPCG_CUDA(cudaMemcpyAsync(h->wsnap.p + (size_t)h->whead * h->ld, a,
                                  sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream));
        h->whead = (h->whead + 1) % h->wq;
        h->wcount = std::min(h->wcount + 1, h->wq);
        KPCG_CUDA(cudaStreamSynchronize(h->stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_warm_fit(kpcg_t h, const double* a, double* c) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        kpcg::check_dev_ptr(a, "a");
        kpcg::check_dev_ptr(c, "c");
        if (h->wmode == 2) {
            kpcg::snapshot_fit(*h, a, c);
            return KPCG_OK;
        }
        ensure_warm(*h);
        kpcg::nystrom_project_solve(h->Wb, a, h->n, 1, c, h->stream);
        KPCG_CUDA(cudaStreamSynchronize(h->stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_warm_expand(kpcg_t h, const double* c, double* x0) {
    if (!h) return KPCG_ERR_ARG;
    KPCG_GUARD(h, {
        kpcg::check_dev_ptr(c, "c");
        kpcg::check_dev_ptr(x0, "x0");
        if (h->wmode == 2) {
            kpcg::snapshot_expand(*h, c, x0);
            return KPCG_OK;
        }
        ensure_warm(*h);
        kpcg::nystrom_expand(h->Wb, c, x0, h->stream);
        KPCG_CUDA(cudaStreamSynchronize(h->stream));
    });
    return KPCG_OK;
}

void kpcg_destroy(kpcg_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->hflags) cudaFreeHost(h->hflags);
    delete h;
}

const char* kpcg_last_error(kpcg_t h) {
    if (!h) return kpcg::g_create_err.c_str();
    return h->err.c_str();
}

}  // extern "C"
