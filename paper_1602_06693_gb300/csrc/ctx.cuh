// Handle state shared by the translation units of libkpcg.
#pragma once

#include <string>
#include <vector>

#include "kpcg_internal.cuh"
#include "precond.cuh"

namespace kpcg {

constexpr double kLog2e = 1.4426950408889634;

template <typename T>
struct CgBufs {
    DevBuf<T> x, r, z, p, q, b;
};

// Device-time accounting of the hot calls (opt.profile): CUDA events around
// each call on the handle's stream, summed when the call returns.
struct Profiler {
    // KV_INNER: reduced-precision products (mixed modes) or the working-precision
    // products (single modes); KV_OUTER: outer direction products; RESID: true
    // residuals (FP64 certification, double-float steering); PRECOND: applies
    enum { KV_INNER = 0, KV_OUTER = 1, PRECOND = 2, RESID = 3, NCAT = 4 };
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans[NCAT];
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        KPCG_CUDA(cudaEventCreate(&e));
        return e;
    }
    template <typename F>
    void time(int cat, cudaStream_t st, F&& f) {
        if (!on) {
            f();
            return;
        }
        cudaEvent_t a = get(), b = get();
        KPCG_CUDA(cudaEventRecord(a, st));
        f();
        KPCG_CUDA(cudaEventRecord(b, st));
        spans[cat].push_back({a, b});
    }
    // Sum and recycle; the stream must have finished.
    void collect(double ms[NCAT], int calls[NCAT]) {
        for (int c = 0; c < NCAT; ++c) {
            ms[c] = 0.0;
            calls[c] = (int)spans[c].size();
            for (auto& s : spans[c]) {
                float t = 0.f;
                if (cudaEventElapsedTime(&t, s.first, s.second) == cudaSuccess) ms[c] += t;
                pool.push_back(s.first);
                pool.push_back(s.second);
            }
            spans[c].clear();
        }
    }
    ~Profiler() {
        for (int c = 0; c < NCAT; ++c)
            for (auto& s : spans[c]) {
                cudaEventDestroy(s.first);
                cudaEventDestroy(s.second);
            }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0, ld = 0;
    int d = 0, dp = 0, ard = 1;
    std::vector<double> log_theta;
    double noise = 0.0, s2 = 1.0;
    kpcg_options opt{};
    DevBuf<float> X;
    DevBuf<double> mu, inv_ell;
    DevBuf<double> xs64;
    DevBuf<float> xs32;
    KvWorkspace kvws;
    PrecondState P;
    CgBufs<double> c64;
    CgBufs<float> c32;
    DevBuf<double> R64, Q64, Bblk, Sblk, G, colscale, fcgP, fcgAP;
    // preconditioner request, replayed when the noise it needs changes
    int pkind = KPCG_PREC_NONE;
    int64_t psize = 0;
    std::vector<int64_t> pidx;
    std::vector<double> pomega;  // spectral draws (m x d) of KPCG_PREC_SPECTRAL
    int64_t pblock = 0;          // block size of KPCG_PREC_PITC
    // warm-start basis (Nystrom-type fit), rebuilt lazily when theta changes
    PrecondState Wb;
    std::vector<int64_t> widx;
    double wridge = 0.0;
    DevBuf<float> W32;
    // snapshot basis: ring of the wq most recent pushed solutions (column-major, ld)
    int wmode = 0;  // 0 none, 1 kernel basis, 2 snapshots
    int wq = 0, wcount = 0, whead = 0;
    DevBuf<double> wsnap, wc;
    DevBuf<double> partial;
    DevBuf<double> scal;
    DevBuf<int> iscal;
    int* hflags = nullptr;  // pinned host [active, broken]
    const int* cg_active = nullptr;  // device flags of the columns the running CG iterates
    bool use_graph = false;          // replay CG iterations from a captured CUDA graph
    std::vector<char> outer_cols;    // during an outer product: columns with a nonzero direction
    // the handle's Nystrom preconditioner as a batch of one problem (FP32 apply of
    // the mixed solve), planned for nys1_c columns and build nys1_version
    NysBatch nys1;
    int nys1_c = -1;
    long long nys1_version = -1;
    long long pversion = 0;  // incremented by every preconditioner build
    // predictions (predict.cu): scaled test inputs, k_* blocks, their solves, partials
    DevBuf<double> pxt, pKb, pW, ppart;
    // Laplace approximation (laplace.cu): P_B, the unscaled K_XU, vectors, CG state
    PrecondState LP;
    DevBuf<float2> lkxu0;
    DevBuf<double> lap;
    CgBufs<double> lcg;
    DevBuf<double> lpw, lpv;  // Laplace predictions: blocks of right-hand sides, variances
    DevBuf<float> lpw32;      // Laplace mixed-precision B-solves: FP32 W^1/2 and scratch
    Profiler prof;
    // tensor-core operands (bf16 bits, pre-swizzled), rebuilt when theta changes
    int theta_version = 0, tc_version = -1, tc_kch = 0;
    DevBuf<uint16_t> tcA, tcB;
    DevBuf<float> tcV, tcPart;
    DevBuf<int> tc_err;
    // tensor-core K.V with the contraction on the tensor cores (kv_tcv_apply;
    // the exponent operands tcA / tcB): V staged as FP16 pairs, partials,
    // per-column max and exponent of V
    DevBuf<uint16_t> tcvV;
    DevBuf<float> tcvPart;
    DevBuf<int> tcvAux;
    // the same product on symmetric tile pairs (kv_tcs.cu): work list, CSR of
    // the items per column tile, staged V, row and column partials
    int tcs_nitems = 0;
    int64_t tcs_n = -1;
    DevBuf<int> tcs_work, tcs_cols;
    DevBuf<float> tcsV, tcsRow, tcsCol;
    // double-float product with sliced tensor-core distances (kv_tcd.cu)
    int tcd_version = -1;
    DevBuf<uint16_t> tcdA, tcdB;
    DevBuf<float2> tcdV;
    DevBuf<double> tcdPart, tcd_max;
    bool df_tensor = true;  // kv_df uses kv_tcd where supported (cleared by tests of the other)
    // its symmetric form (one evaluation per pair of points): B in 32-row
    // tiles, the work list, row and column partials
    bool tcd_symmetric = true;  // cleared by the tests of the one-sided kernel
    int tcds_version = -1, tcds_nitems = 0;
    int64_t tcds_n = -1;
    DevBuf<uint16_t> tcdBs;
    DevBuf<int> tcds_work, tcds_rows;
    DevBuf<double> tcdsRow, tcdsCol;
    // per-point-exact tensor-core operands (kv_tcx_apply), rebuilt when theta changes
    int tcx_version = -1, tcx_kch = 0, tcx_nmma = 0;
    float tcx_escale = 1.f;
    DevBuf<uint16_t> tcxA, tcxB;
    DevBuf<double> tcxPart, tcx_max;
    // double-float operands (kv_df.cu), rebuilt when theta changes
    int df_version = -1;
    float df_c0h = 0.f, df_c0l = 0.f;
    DevBuf<float> xdf;
    DevBuf<float> xf2;  // (hi, lo) pairs of x' for the exact-difference FP32 kernel
    DevBuf<float2> df_tab, df_tab1k;
    DevBuf<double> f64_tab;  // 2^(j/256) for the table-driven FP64 exp of kv_f64_sym
    DevBuf<double> df_grid;
    bool df_symmetric = true;  // symmetric tile-pair kernel (cleared by tests of the other)
    int64_t df_sym_n = -1;
    int df_sym_G = 0, df_nwork = 0;
    DevBuf<int> df_work;
    DevBuf<double> df_prow, df_pcol;
    std::string err;

    double c0_64() const { return std::log(s2); }
    float c0_32() const { return (float)(std::log(s2) * kLog2e); }
};

// Tensor-core K.V on the handle's inputs (kv_tc.cu).
void kv_tc_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo, float noise);
// O = K V + noise V (or B - that when B != nullptr) with the double-float
// kernel (kv_df.cu); FP64 in and out.
void kv_df(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb, double* O,
           int64_t ldo, double noise);
// Native-FP64 product on symmetric tile pairs (kv_df.cu); falls back to the
// row-split kernel for small n or d > 16.  Same arguments as kv_df.
void kv_f64_sym(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb,
                double* O, int64_t ldo, double noise);
// O = (K + noise I) V in FP32 with exact pairwise differences of the split
// inputs and compensated sums (kv_df.cu; d <= 16).  expp 0: MUFU exp2,
// 1: polynomial exp2 on the FMA pipe.
void kv_xf(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo, float noise,
           int expp);
bool kv_xf_supported(const Ctx& h);
// dK/dtheta_q W (FP64 in and out) in double-float arithmetic (kv_df.cu;
// d <= 16); layout of kpcg_dkv.
void dkv_df(Ctx& h, const double* W, int64_t ldw, int c, double* G, int64_t ldg);
// Tensor-core K.V on per-point-exact sliced operands (kv_tc.cu; d <= 10):
// FP32 in and out, FP32 exponent rounding relative to the exponent itself,
// compensated row sums.
void kv_tcx_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  float noise);
bool kv_tcx_supported(int d);
// The same product for FP64 vectors (V staged as FP32 pairs, FP64 out).
void kv_tcx_apply64(Ctx& h, const double* V, int64_t ldv, int c, double* O, int64_t ldo,
                    double noise);
// Nonzero if a bounded wait inside the tensor-core kernel expired since the
// last call (the flag is cleared).
int kv_tc_error(Ctx& h);
int sm_count_tc();
// Operands of the tensor-core products for the handle's current theta (kv_tc.cu).
void tc_prepare(Ctx& h);
// Tensor-core K.V with the second contraction on the tensor cores as well
// (kv_tcv.cu; d <= 20): FP32 in and out, the exponentiated tile as FP16
// pairs in tensor memory against V as FP16 pairs.
void kv_tcv_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  float noise);
bool kv_tcv_supported(int d);
// Double-float K.V (FP64 in and out, arguments of kv_df) with the squared
// distances from exact integer level sums on the tensor cores (kv_tcd.cu;
// d <= 10); the exp2 and the contraction in double-float on the FP32 pipe.
void kv_tcd(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb, double* O,
            int64_t ldo, double noise);
bool kv_tcd_supported(const Ctx& h);
// Double-float inputs of the handle (exp2 table, log2(s^2) pair), kv_df.cu.
void df_prepare(Ctx& h);
// Column count from which the inner products of the mixed solvers use
// kv_tcv_apply: below it the FP32-FMA contraction of kv_tc_apply costs less
// issue per entry than the FP16 split of the tile, above it more.
constexpr int kTcvMinCols = 4;
// Tensor-core K.V (the entries of kv_tc_apply) on symmetric tile pairs, one
// column at a time (kv_tcs.cu); usable for n > 128 and d <= 20.
void kv_tcs_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  float noise);
bool kv_tcs_usable(const Ctx& h);
// The tensor-core inner product of the mixed solvers for c columns.
inline void kv_tc_inner(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                        float noise) {
    if (c >= kTcvMinCols && kv_tcv_supported(h.d))
        kv_tcv_apply(h, V, ldv, c, O, ldo, noise);
    else if (kv_tcs_usable(h))
        kv_tcs_apply(h, V, ldv, c, O, ldo, noise);
    else
        kv_tc_apply(h, V, ldv, c, O, ldo, noise);
}

}  // namespace kpcg

// The opaque handle of the C ABI.
struct kpcg_ctx : kpcg::Ctx {};
