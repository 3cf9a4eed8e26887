// Solver pieces shared by the single-problem handle (api.cu) and the batch
// of uneven problems (batch.cu).
#pragma once

#include <functional>
#include <vector>

#include "ctx.cuh"

namespace kpcg {

// The operators of the mixed-precision solve: the flexible-CG outer loop in
// FP64 (Notay's FCG around an inexact inner solve, Sec. 3.3.2) only sees
// these, so one loop serves one problem or a batch laid out column by column.
struct MixedOps {
    // O = (K + inner noise I) V in FP32, and the inner preconditioner
    std::function<void(const float*, int64_t, int, float*, int64_t)> inner_mv, inner_pc;
    // when set: the inner PCG runs on FP64 vectors with these instead
    std::function<void(const double*, int64_t, int, double*, int64_t)> inner_mv64, inner_pc64;
    // O = K_y V with FP64-class accuracy
    std::function<void(const double*, int64_t, int, double*, int64_t)> outer_mv;
    // R = B - K_y X and the per-column ||R||^2, ||B||^2; certify: native FP64
    // (the value the stop test is decided on), else FP64-class (steering only)
    std::function<void(const double*, int64_t, int, const double*, int64_t, double*,
                       std::vector<double>&, std::vector<double>&, bool certify)>
        residual;
    // true if a bounded device wait expired since the last query
    std::function<bool()> timed_out;
};

// Makes the active-column flags of the running CG visible to the operators
// (h.cg_active) for the lifetime of one pcg_core call.
struct ActiveScope {
    Ctx& h;
    const int* saved;
    ActiveScope(Ctx& hh, const int* a) : h(hh), saved(hh.cg_active) { h.cg_active = a; }
    ~ActiveScope() { h.cg_active = saved; }
};

// One captured chunk of CG iterations.  capture(h, f) records f(cs) on a
// private non-blocking stream cs (the handle's stream may be the legacy
// default stream, which cannot be captured) while h.stream points at cs, so
// operators that launch on h.stream are recorded too; the graph is then
// launched on the handle's own stream.
struct GraphChunk {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;  // kernel launches recorded, counted again per replay
    template <typename F>
    void capture(Ctx& h, F&& f) {
        const long long l0 = launch_count();
        cudaStream_t cs = nullptr;
        KPCG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaStream_t saved = h.stream;
        h.stream = cs;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            try {
                f(cs);
            } catch (...) {
                cudaStreamEndCapture(cs, &g);
                if (g) cudaGraphDestroy(g);
                h.stream = saved;
                cudaStreamDestroy(cs);
                throw;
            }
            e = cudaStreamEndCapture(cs, &g);
        }
        h.stream = saved;
        cudaStreamDestroy(cs);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        KPCG_CUDA(e);
        // the recording launched nothing: take those counts back, replays add them
        kernels = launch_count() - l0;
        note_launches(-kernels);
    }
    ~GraphChunk() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

kpcg_status fcg_solve(Ctx& h, const MixedOps& ops, const double* B, int64_t ldb, int c,
                      double tol, const double* X0, double* Xout, int64_t ldx,
                      std::vector<int>& iters_col, int& iters_total, int& steps,
                      std::vector<double>& rr, std::vector<double>& bb);
bool col_converged(double rr, double bb, double tol, int tol_mode, int64_t n);
// O = A V for c columns (ld-strided, column-major); must launch on h.stream
using VecOp = std::function<void(const double*, int64_t, int, double*, int64_t)>;
// Column-wise PCG (Algorithm 1) in FP64 on an operator and preconditioner of
// the caller's (relative stop test ||r|| <= tol ||b|| per column, on the
// recursive residual); X holds x0 unless x0_zero.  Returns the iterations run.
int pcg_f64(Ctx& h, int c, const double* B, int64_t ldb, double* X, int64_t ldx, bool x0_zero,
            double tol, int max_iter, const VecOp& matvec, const VecOp& precond,
            CgBufs<double>& bufs, std::vector<int>& iters, int& broken);
// The solve behind kpcg_solve: K_y X = B for c columns with the handle's
// precision and preconditioner (device blocks; iters_host, info nullable).
kpcg_status solve_impl(Ctx& h, const double* B, int64_t ldb, int c, double tol,
                       const double* X0, double* Xout, int64_t ldx, int32_t* iters_host,
                       kpcg_info* info);
// Predictions (predict.cu): scale Xs (ns x d row-major, float32) into the
// handle's coordinates (kept in c.pxt, returned) and write mean = K(X_*, X) alpha
// (FP64); and the block K(X, X_*) of nb scaled test points into Kb (ld ldk).
const double* predict_mean(Ctx& c, const float* Xs, int64_t ns, const double* alpha,
                           double* mean);
void predict_kblock(Ctx& c, const double* xt, int nb, double* Kb, int64_t ldk);
// (Re)build the handle's preconditioner for the noise its mode needs;
// returns the host milliseconds spent (0 if it was current).
double ensure_precond(Ctx& h);

}  // namespace kpcg
