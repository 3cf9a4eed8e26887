// Many independent GP systems of uneven size solved together: one handle per
// problem holds its inputs, theta and Nystrom preconditioner; the batch lays
// every (problem, right-hand side) pair out as one column of a shared block
// (batch.cuh) and runs the mixed-precision solve over all of them at once:
// flexible CG in FP64 outside, FP32 PCG inside, where every inner product
// with K is one persistent tensor-core launch over the flat tile list of all
// problems and every preconditioner apply is one batched launch sequence.
// The outer loop's direction products use the double-float kernel per
// problem and every true residual the native-FP64 one (its error scales with
// the full solution, the directions' with the small correction).  Columns,
// hence problems, stop independently.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "batch.cuh"
#include "solver.cuh"

namespace kpcg {
namespace {

// dst[:, p*c + k] = src[:, p*c + k] on rows < n_p, zero on rows n_p .. nrows-1.
template <typename TD, typename TS>
__global__ void masked_copy_kernel(TD* __restrict__ dst, int64_t ldd, const TS* __restrict__ src,
                                   int64_t lds, const int64_t* __restrict__ nrow, int c,
                                   int64_t nrows) {
    const int col = blockIdx.y;
    const int64_t np = nrow[col / c];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i + (int64_t)col * ldd] = (i < np) ? (TD)src[i + (int64_t)col * lds] : (TD)0;
}

}  // namespace
}  // namespace kpcg

using kpcg::fail;

struct kpcg_batch {
    std::vector<kpcg_ctx*> sub;
    kpcg::Ctx M;  // CG buffers and options of the whole block; n = max n_p
    int64_t nmax = 0;
    kpcg::DevBuf<int64_t> nrow;  // n_p per problem (device)
    kpcg::TcBatch tc;
    int tc_G = 0, tc_grid = 0;   // 0: autotune at the first product
    int tc_tcv = -1;             // contraction on the tensor cores (-1: not chosen yet)
    int tcv_mode = -1;           // the caller's choice of it (-1: autotuner / column count)
    float tuned_ms = 0.f;
    kpcg::NysBatch nys;
    kpcg::DevBuf<double> Bp, Xp;
    std::string err;
};

namespace kpcg {
namespace {

std::vector<float> inner_noise(const kpcg_batch& b) {
    std::vector<float> v;
    for (auto* h : b.sub) v.push_back((float)(h->noise * (1.0 + b.M.opt.inner_shift)));
    return v;
}
std::vector<Ctx*> subs_of(const kpcg_batch& b) {
    return std::vector<Ctx*>(b.sub.begin(), b.sub.end());
}

// Time the batched product for each candidate run length (tiles per work
// item) and each contraction path (FP32 FMAs on pairs of row tiles, or the
// tensor cores) and keep the fastest; the grid is one persistent CTA per SM
// (the kernels' shared memory admits one).
void autotune(kpcg_batch& b, int c) {
    cudaStream_t st = b.M.stream;
    const int64_t ld = b.M.ld;
    const int P = (int)b.sub.size();
    float* V = b.M.c32.b.need((size_t)ld * P * c);
    float* O = b.M.c32.q.need((size_t)ld * P * c);
    KPCG_CUDA(cudaMemsetAsync(V, 0, sizeof(float) * (size_t)ld * P * c, st));
    const auto noise = inner_noise(b);
    const auto subs = subs_of(b);
    cudaEvent_t e0, e1;
    KPCG_CUDA(cudaEventCreate(&e0));
    KPCG_CUDA(cudaEventCreate(&e1));
    int bestG = 8, bestV = 0;
    b.tc_tcv = -1;
    float best = INFINITY;
    bool tcv_ok = true;
    for (auto* h : b.sub) tcv_ok = tcv_ok && kv_tcv_supported(h->d);
    const int tcv_lo = b.tcv_mode >= 0 ? b.tcv_mode : 0;
    const int tcv_hi = b.tcv_mode >= 0 ? b.tcv_mode : (tcv_ok ? 1 : 0);
    for (int tcv = tcv_lo; tcv <= tcv_hi; ++tcv)
    for (int G : {1, 2, 4, 8, 16, 32, 64}) {
        tc_batch_plan(b.tc, subs, noise, G, 0, st, tcv);
        kv_tc_batch(b.tc, V, ld, c, O, ld, b.M.n, nullptr, st);  // warm-up
        KPCG_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) kv_tc_batch(b.tc, V, ld, c, O, ld, b.M.n, nullptr, st);
        KPCG_CUDA(cudaEventRecord(e1, st));
        KPCG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        KPCG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 3.f;
        if (ms < best) {
            best = ms;
            bestG = G;
            bestV = tcv;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (kv_tc_batch_error(b.tc, st)) fail(KPCG_ERR_TIMEOUT, "a bounded wait in the batched K.V expired");
    b.tc_G = bestG;
    b.tc_grid = sm_count_tc();
    b.tc_tcv = bestV;
    b.tuned_ms = best;
}

void ensure_tc(kpcg_batch& b, int c) {
    if (b.tc_G == 0) autotune(b, c);
    if (b.tcv_mode >= 0) b.tc_tcv = b.tcv_mode;
    if (b.tc_tcv < 0) {  // a tiling fixed by the caller: the path by the column count
        bool ok = true;
        for (auto* h : b.sub) ok = ok && kv_tcv_supported(h->d);
        b.tc_tcv = (ok && c >= 4) ? 1 : 0;
    }
    tc_batch_plan(b.tc, subs_of(b), inner_noise(b), b.tc_G, b.tc_grid, b.M.stream, b.tc_tcv);
}

void ensure_nys(kpcg_batch& b, int c) {
    std::vector<const PrecondState*> Ps;
    for (auto* h : b.sub) {
        ensure_precond(*h);
        Ps.push_back(&h->P);
    }
    nys_batch_plan(b.nys, Ps, c, b.M.stream);
}

void check_batch_block(const kpcg_batch& b, const void* p, int64_t ld, int c, const char* name) {
    if (!p) fail(KPCG_ERR_ARG, std::string(name) + " is NULL");
    if (ld < b.nmax) fail(KPCG_ERR_ARG, std::string(name) + ": leading dimension below max n");
    if (c < 1) fail(KPCG_ERR_ARG, "c must be >= 1");
    if ((int64_t)c * (int64_t)b.sub.size() > 65535)
        fail(KPCG_ERR_ARG, "nprob * c must be <= 65535");
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        fail(KPCG_ERR_ARG, std::string(name) + " must be device memory");
    }
}

}  // namespace
}  // namespace kpcg

#define BATCH_GUARD(bp, ...)                                 \
    try {                                                    \
        __VA_ARGS__;                                         \
    } catch (const kpcg::Error& e) {                         \
        if (bp) (bp)->err = e.msg;                           \
        else kpcg::set_handleless_error(e.msg);              \
        return e.status;                                     \
    }

extern "C" {

kpcg_status kpcg_batch_create(int32_t nprob, const kpcg_problem* probs, const kpcg_options* opt,
                              void* stream, kpcg_batch_t* out) {
    kpcg_batch* b = nullptr;
    try {
        if (!out || !probs) fail(KPCG_ERR_ARG, "NULL argument");
        *out = nullptr;
        if (nprob < 1 || nprob > 4096) fail(KPCG_ERR_ARG, "nprob must be in [1, 4096]");
        kpcg_options o;
        kpcg_default_options(&o);
        o.precision = KPCG_TC_IR;
        if (opt) {
            o = *opt;
            if (o.precision != KPCG_TC_IR)
                fail(KPCG_ERR_ARG, "batch solves run the tensor-core mixed-precision mode");
        }
        b = new kpcg_batch();
        b->M.stream = (cudaStream_t)stream;
        KPCG_CUDA(cudaGetDevice(&b->M.device));
        std::vector<int64_t> nr;
        for (int p = 0; p < nprob; ++p) {
            const kpcg_problem& q = probs[p];
            if (q.d > 16) fail(KPCG_ERR_ARG, "batch problems need d <= 16");
            kpcg_t h = nullptr;
            const kpcg_status st =
                kpcg_create(q.X, q.n, q.d, q.log_theta, q.ard, q.noise_var, &o, stream, &h);
            if (st != KPCG_OK)
                fail(st, "problem " + std::to_string(p) + ": " + kpcg_last_error(nullptr));
            b->sub.push_back(h);
            if (q.m > 0) {
                const kpcg_status s2 = kpcg_precond(h, KPCG_PREC_NYSTROM, q.m, q.idx);
                if (s2 != KPCG_OK)
                    fail(s2, "problem " + std::to_string(p) + ": " + kpcg_last_error(h));
            }
            nr.push_back(q.n);
            b->nmax = std::max(b->nmax, q.n);
        }
        b->M.n = b->nmax;
        b->M.ld = ((b->nmax + 127) / 128) * 128;
        b->M.opt = o;
        b->M.d = 1;
        b->M.use_graph = true;
        KPCG_CUDA(cudaHostAlloc((void**)&b->M.hflags, 4 * sizeof(int), cudaHostAllocDefault));
        b->nrow.need(nr.size());
        KPCG_CUDA(cudaMemcpyAsync(b->nrow.p, nr.data(), sizeof(int64_t) * nr.size(),
                                  cudaMemcpyHostToDevice, b->M.stream));
        KPCG_CUDA(cudaStreamSynchronize(b->M.stream));
        *out = b;
        return KPCG_OK;
    } catch (const kpcg::Error& e) {
        kpcg::set_handleless_error(e.msg);
        if (b) kpcg_batch_destroy(b);
        return e.status;
    }
}

int64_t kpcg_batch_max_n(kpcg_batch_t b) { return b ? b->nmax : 0; }

kpcg_status kpcg_batch_set_options(kpcg_batch_t b, const kpcg_options* opt) {
    if (!b) return KPCG_ERR_ARG;
    BATCH_GUARD(b, {
        if (!opt) fail(KPCG_ERR_ARG, "opt is NULL");
        if (opt->precision != KPCG_TC_IR)
            fail(KPCG_ERR_ARG, "batch solves run the tensor-core mixed-precision mode");
        for (auto* h : b->sub) {
            const kpcg_status st = kpcg_set_options(h, opt);
            if (st != KPCG_OK) fail(st, kpcg_last_error(h));
        }
        b->M.opt = *opt;
    });
    return KPCG_OK;
}

kpcg_status kpcg_batch_set_tiling(kpcg_batch_t b, int32_t tiles_per_item, int32_t ctas) {
    if (!b) return KPCG_ERR_ARG;
    BATCH_GUARD(b, {
        if (tiles_per_item < 1 || ctas < 0) fail(KPCG_ERR_ARG, "bad tiling");
        b->tc_G = tiles_per_item;
        b->tc_grid = ctas;
    });
    return KPCG_OK;
}

kpcg_status kpcg_batch_set_contraction(kpcg_batch_t b, int32_t mode) {
    if (!b) return KPCG_ERR_ARG;
    BATCH_GUARD(b, {
        if (mode < -1 || mode > 1) fail(KPCG_ERR_ARG, "mode must be -1, 0 or 1");
        if (mode == 1)
            for (auto* h : b->sub)
                if (!kpcg::kv_tcv_supported(h->d))
                    fail(KPCG_ERR_ARG, "the tensor-core contraction supports d <= 20");
        b->tcv_mode = mode;
        b->tc_tcv = mode;
    });
    return KPCG_OK;
}

kpcg_status kpcg_batch_tune(kpcg_batch_t b, int32_t c, int32_t* tiles_per_item, int32_t* ctas,
                            float* best_ms) {
    if (!b) return KPCG_ERR_ARG;
    BATCH_GUARD(b, {
        if (c < 1) fail(KPCG_ERR_ARG, "c must be >= 1");
        kpcg::autotune(*b, c);
        if (tiles_per_item) *tiles_per_item = b->tc_G;
        if (ctas) *ctas = b->tc_grid;
        if (best_ms) *best_ms = b->tuned_ms;
    });
    return KPCG_OK;
}

kpcg_status kpcg_batch_matvec_f32(kpcg_batch_t b, const float* V, int64_t ld, int32_t c, float* O) {
    if (!b) return KPCG_ERR_ARG;
    BATCH_GUARD(b, {
        kpcg::check_batch_block(*b, V, ld, c, "V");
        kpcg::check_batch_block(*b, O, ld, c, "O");
        kpcg::ensure_tc(*b, c);
        kpcg::kv_tc_batch(b->tc, V, ld, c, O, ld, b->nmax, nullptr, b->M.stream);
        KPCG_CUDA(cudaStreamSynchronize(b->M.stream));
        if (kpcg::kv_tc_batch_error(b->tc, b->M.stream))
            fail(KPCG_ERR_TIMEOUT, "a bounded wait in the batched K.V expired");
    });
    return KPCG_OK;
}

kpcg_status kpcg_batch_precond_apply_f32(kpcg_batch_t b, const float* R, int64_t ld, int32_t c,
                                         float* Z) {
    if (!b) return KPCG_ERR_ARG;
    BATCH_GUARD(b, {
        kpcg::check_batch_block(*b, R, ld, c, "R");
        kpcg::check_batch_block(*b, Z, ld, c, "Z");
        kpcg::ensure_nys(*b, c);
        kpcg::nys_batch_apply(b->nys, R, ld, Z, ld, b->nmax, nullptr, b->M.stream);
        KPCG_CUDA(cudaStreamSynchronize(b->M.stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_batch_solve(kpcg_batch_t b, const double* B, int64_t ld, int32_t c, double tol,
                             double* X, int32_t* iters, double* rel_res, kpcg_info* info) {
    if (!b) return KPCG_ERR_ARG;
    kpcg_status status = KPCG_OK;
    BATCH_GUARD(b, {
        using namespace kpcg;
        const auto t0 = std::chrono::steady_clock::now();
        const long long launches0 = launch_count();
        check_batch_block(*b, B, ld, c, "B");
        check_batch_block(*b, X, ld, c, "X");
        if (!(tol > 0.0)) fail(KPCG_ERR_ARG, "tol must be > 0");
        Ctx& M = b->M;
        cudaStream_t st = M.stream;
        const int P = (int)b->sub.size();
        const int C = P * c;
        const int64_t L = M.ld;
        M.prof.on = (M.opt.profile != 0);
        const auto ts = std::chrono::steady_clock::now();
        ensure_nys(*b, c);
        ensure_tc(*b, c);
        const double setup_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts)
                .count();
        // padded copies and zeroed work blocks: rows n_p .. of every column stay zero
        const int W = std::max(1, M.opt.fcg_window);
        double* Bp = b->Bp.need((size_t)L * C);
        double* Xp = b->Xp.need((size_t)L * C);
        const dim3 g((unsigned)std::min<int64_t>((L + 255) / 256, 64), (unsigned)C);
        masked_copy_kernel<double, double><<<g, 256, 0, st>>>(Bp, L, B, ld, b->nrow.p, c, L);
        KPCG_LAUNCHED("masked_copy_kernel");
        auto zero = [&](auto& buf, size_t count) {
            auto* p = buf.need(count);
            KPCG_CUDA(cudaMemsetAsync(p, 0, sizeof(*p) * count, st));
        };
        zero(M.R64, (size_t)L * C);
        zero(M.Q64, (size_t)L * C);
        zero(M.fcgP, (size_t)W * L * C);
        zero(M.fcgAP, (size_t)W * L * C);
        zero(M.c32.b, (size_t)L * C);
        zero(M.c32.x, (size_t)L * C);

        MixedOps ops;
        kpcg_batch* bb = b;
        ops.inner_mv = [bb, c](const float* V, int64_t ldv, int, float* O, int64_t ldo) {
            kv_tc_batch(bb->tc, V, ldv, c, O, ldo, bb->M.n, bb->M.cg_active, bb->M.stream);
        };
        ops.inner_pc = [bb](const float* R, int64_t ldr, int, float* Z, int64_t ldz) {
            nys_batch_apply(bb->nys, R, ldr, Z, ldz, bb->M.n, bb->M.cg_active, bb->M.stream);
        };
        ops.outer_mv = [bb, c](const double* V, int64_t ldv, int, double* O, int64_t ldo) {
            const auto& live = bb->M.outer_cols;
            for (size_t p = 0; p < bb->sub.size(); ++p) {
                Ctx& h = *bb->sub[p];
                const int64_t off = (int64_t)p * c;
                bool any = live.empty();
                for (int k = 0; k < c && !any; ++k) any = live[(size_t)off + k] != 0;
                if (!any) {  // every direction of this problem is zero: so is K_y p
                    KPCG_CUDA(cudaMemsetAsync(O + off * ldo, 0, sizeof(double) * (size_t)c * ldo,
                                              bb->M.stream));
                    continue;
                }
                kv_df(h, V + off * ldv, ldv, c, nullptr, 0, O + off * ldo, ldo, h.noise);
            }
        };
        ops.residual = [bb, c](const double* Bm, int64_t ldb, int cc, const double* Xm, int64_t ldx,
                               double* R, std::vector<double>& rr, std::vector<double>& bn,
                               bool certify) {
            Ctx& M = bb->M;
            for (size_t p = 0; p < bb->sub.size(); ++p) {
                Ctx& h = *bb->sub[p];
                const int64_t off = (int64_t)p * c;
                // certify: native FP64 (b - K x cancels terms up to ~|x|/|b| ~
                // 1/sigma^2 larger than the result, beyond the double-float
                // product's reach); steering only: double-float
                M.prof.time(Profiler::RESID, M.stream, [&] {
                    if (certify)
                        kv_f64(h.xs64.p, h.n, h.dp, h.c0_64(), h.noise, Xm + off * ldx, ldx, c,
                               Bm + off * ldb, ldb, R + off * M.ld, M.ld, h.kvws, M.stream);
                    else
                        kv_df(h, Xm + off * ldx, ldx, c, Bm + off * ldb, ldb, R + off * M.ld,
                              M.ld, h.noise);
                });
            }
            const int nblk = dot_blocks(M.n);
            double* partial = M.partial.need((size_t)nblk * cc * 2);
            dot_cols<double>(R, M.ld, R, M.ld, M.n, cc, partial, nblk, M.stream);
            dot_cols<double>(Bm, ldb, Bm, ldb, M.n, cc, partial + (size_t)nblk * cc, nblk,
                             M.stream);
            std::vector<double> hp((size_t)nblk * cc * 2);
            KPCG_CUDA(cudaMemcpyAsync(hp.data(), partial, sizeof(double) * hp.size(),
                                      cudaMemcpyDeviceToHost, M.stream));
            KPCG_CUDA(cudaStreamSynchronize(M.stream));
            rr.assign(cc, 0.0);
            bn.assign(cc, 0.0);
            for (int k = 0; k < cc; ++k)
                for (int q = 0; q < nblk; ++q) {
                    rr[k] += hp[(size_t)k * nblk + q];
                    bn[k] += hp[(size_t)(cc + k) * nblk + q];
                }
        };
        ops.timed_out = [bb]() { return kv_tc_batch_error(bb->tc, bb->M.stream) != 0; };

        std::vector<int> iters_col((size_t)C, 0);
        int iters_total = 0, steps = 0;
        std::vector<double> rr, bn;
        // The outer loop gives up when its worst column stops improving; with
        // hundreds of columns of very different difficulty that can be one slow
        // problem in a slow phase.  Restart it from the current iterate (fresh
        // residual, empty direction window) while restarts keep improving.
        double prev_worst = INFINITY;
        for (int restart = 0;; ++restart) {
            int st_steps = 0;
            status = fcg_solve(M, ops, Bp, L, C, tol, restart ? Xp : nullptr, Xp, L, iters_col,
                               iters_total, st_steps, rr, bn);
            steps += st_steps;
            if (status != KPCG_ERR_NO_CONVERGENCE || restart >= M.opt.max_restarts ||
                iters_total >= M.opt.max_iter)
                break;
            double worst = 0.0;
            for (int k = 0; k < C; ++k)
                if (bn[k] > 0) worst = std::max(worst, std::sqrt(rr[k] / bn[k]));
            if (!(worst < 0.5 * prev_worst)) break;
            prev_worst = worst;
        }
        if (status != KPCG_OK) ops.residual(Bp, L, C, Xp, L, M.R64.p, rr, bn, true);
        // exactly ld rows per column of the caller's block (ld may be below L)
        masked_copy_kernel<double, double><<<g, 256, 0, st>>>(X, ld, Xp, L, b->nrow.p, c, ld);
        KPCG_LAUNCHED("masked_copy_kernel");
        double maxrel = 0.0;
        for (int k = 0; k < C; ++k) {
            const double rel = bn[k] > 0 ? std::sqrt(rr[k] / bn[k]) : 0.0;
            maxrel = std::max(maxrel, rel);
            if (rel_res) rel_res[k] = rel;
            if (iters) iters[k] = iters_col[k];
        }
        KPCG_CUDA(cudaStreamSynchronize(st));
        double ms[Profiler::NCAT];
        int calls[Profiler::NCAT];
        M.prof.collect(ms, calls);
        if (info) {
            info->iters_total = iters_total;
            info->outer_steps = steps;
            info->max_rel_res = maxrel;
            info->time_ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count();
            info->setup_ms = setup_ms;
            info->kv_inner_ms = ms[Profiler::KV_INNER];
            info->kv_inner_calls = calls[Profiler::KV_INNER];
            info->kv_outer_ms = ms[Profiler::KV_OUTER];
            info->kv_outer_calls = calls[Profiler::KV_OUTER];
            info->precond_ms = ms[Profiler::PRECOND];
            info->precond_calls = calls[Profiler::PRECOND];
            info->resid_ms = ms[Profiler::RESID];
            info->resid_calls = calls[Profiler::RESID];
            info->launches = (int)(launch_count() - launches0);
            double jit = 0.0;
            for (auto* h : b->sub) jit = std::max(jit, h->P.ready ? h->P.jitter : 0.0);
            info->precond_jitter = jit;
        }
        if (status != KPCG_OK)
            b->err = std::string(kpcg_status_string(status)) + ": max relative residual " +
                     std::to_string(maxrel);
    });
    return status;
}

void kpcg_batch_destroy(kpcg_batch_t b) {
    if (!b) return;
    if (b->M.stream) cudaStreamSynchronize(b->M.stream);
    for (auto* h : b->sub) kpcg_destroy(h);
    if (b->M.hflags) cudaFreeHost(b->M.hflags);
    b->M.hflags = nullptr;
    delete b;
}

const char* kpcg_batch_last_error(kpcg_batch_t b) {
    if (!b) return kpcg_last_error(nullptr);
    return b->err.c_str();
}

}  // extern "C"
