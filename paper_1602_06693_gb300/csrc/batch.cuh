// Many independent kernel systems of uneven size solved together
// (kv_tc.cu: batched tensor-core K.V; precond.cu: batched Nystrom apply;
// batch.cu: the solver and the C ABI).
//
// Layout.  Problem p with n_p rows and c right-hand sides owns columns
// p*c .. p*c+c-1 of every batch vector, an ld x (P c) column-major block with
// ld >= max_p n_p; rows n_p .. ld-1 of its columns are zero and stay zero.
// Every (problem, column) pair is therefore an ordinary column to the CG
// kernels, with its own alpha, beta and stop test (Algorithm 1 per column).
#pragma once

#include <vector>

#include "ctx.cuh"

namespace kpcg {

// ---------------------------------------------------------------- K.V
struct TcBatchProb {
    const uint16_t* A;  // augmented BF16 operands (tc_prepare), pre-swizzled
    const uint16_t* B;
    int64_t voff;       // first row of the problem in the staged V / partial rows
    int32_t n, n_pad, kch, rt_base;
    float noise;        // diagonal added by the product
    float s2;           // signal variance (the tensor-core contraction's output scale)
};
// Column tiles [jt0, jt0 + nt) against row tile rt of problem prob and, if
// two, row tile rt + 1 as well (the epilogue then uses every value of V it
// reads for two rows).
struct TcBatchItem {
    int32_t prob, rt, jt0, nt, two, pad_;
};

struct TcBatch {
    int P = 0, G = 0, grid = 0, nitems = 0;
    // tcv: the second contraction on the tensor cores too (kv_tcv.cu): one row
    // tile per item, V staged as FP16 pairs in Vh,
    // per (problem, column) max |V| and exponent in aux
    int tcv = 0;
    int64_t nv = 0;  // sum of the padded sizes
    std::vector<TcBatchProb> hprobs;
    DevBuf<TcBatchProb> probs;
    DevBuf<TcBatchItem> items;
    DevBuf<int32_t> rt_first, rt_count;  // per (problem, row-tile pair or row tile): its items
    DevBuf<float> Vs, part;
    DevBuf<uint16_t> Vh;
    DevBuf<int> aux;
    DevBuf<int> err;
};

// Operands of the tensor-core product for the handle's current theta.
void tc_prepare(Ctx& h);
int sm_count_tc();
// Work list: every row tile of every problem, its column tiles cut into
// items of at most G tiles; grid = CTAs of the persistent launch (0: one per SM).
// tcv: the kernel with the contraction on the tensor cores (single row tiles).
void tc_batch_plan(TcBatch& b, const std::vector<Ctx*>& subs, const std::vector<float>& noise,
                   int G, int grid, cudaStream_t st, int tcv = 0);
// Operands of kv_tcv_apply for the handle's current theta (kv_tcv.cu: those
// of tc_prepare, after the dimension check of the tcv path).
void tcv_prepare(Ctx& h);
// The tcv batched product (kv_tcv.cu); called by kv_tc_batch when b.tcv is set.
void kv_tcv_batch(TcBatch& b, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  int64_t nrows, const int* active, cudaStream_t st);
// O = (K_p + noise_p I) V for every problem (columns p*c ..), rows n_p .. nrows-1
// of O set to zero.  active (nullable, P*c flags): problems with no active
// column are skipped and their columns of O set to zero.
void kv_tc_batch(TcBatch& b, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                 int64_t nrows, const int* active, cudaStream_t st);
// Nonzero if a bounded wait of the batched kernel expired (flag cleared).
int kv_tc_batch_error(TcBatch& b, cudaStream_t st);

}  // namespace kpcg
