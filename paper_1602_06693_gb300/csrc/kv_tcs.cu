// Tensor-core K.V on symmetric tile pairs, FP32 (the inner product of the
// mixed-precision solver, KPCG_TC_IR, for one column at a time).
//
// The entries are those of kv_tc_kernel: the BF16x3 augmented operands of
// tc_prep_kernel give the exp2 argument a_ij = log2(s^2) - |x'_i - x'_j|^2 of
// Eq. 1 in an FP32 accumulator, exp2 runs on the MUFU.  K is symmetric, so
// each pair of 128-point tiles (I, J), I <= J, is evaluated once: the tile
// gives the row sums K_IJ V_J for the rows of I and, from the same entries,
// the column sums K_IJ^T V_I for the rows of J (not for I = J, whose tile is
// evaluated in full and gives row sums only).
//
// The column tile J is the CTA's resident operand (B in shared memory for the
// whole work item, its V_J in registers) and the row tiles I stream through a
// ring (A tile and V_I per stage).  Each epilogue thread owns one row of the
// tile and 64 of its columns: per entry one TMEM word, one ex2, one FMA into
// its row sum (V_j from registers) and one FMA into its column accumulator
// (V_i, one value per tile) -- no shared-memory traffic and no shuffles per
// entry.  The column accumulators are reduced over the 128 rows once per work
// item (a shuffle butterfly, then the four row quarters through shared
// memory).  Row sums leave once per tile pair and half, column sums once per
// work item; a second kernel adds, for every point, its row partials and the
// column partials of its tile in a fixed order, in FP64.
//
// Roles (10 warps, one CTA per SM): warp 0 bulk-copies (the B tile once, then
// A tiles and V_I into a 4-stage ring), warp 1 issues the MMAs from one
// thread into double-buffered TMEM accumulators, warps 2..9 are the epilogue
// (row quarter = warp mod 4, the TMEM lanes a warp may read; column half =
// (warp - 2) / 4).  Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "tcgen05.cuh"

namespace kpcg {
namespace {

constexpr int SWARPS_TCS = 10;
constexpr int SEPI_TCS = 8;
constexpr int STAGES_TCS = 4;

template <int KCH>
struct TcsSmem {
    static constexpr uint32_t kSub = SUB * 2;                           // 16 KB
    static constexpr uint32_t kB = KCH * kSub;                          // resident B tile
    static constexpr uint32_t kAst = KCH * kSub;                        // A part of a stage
    static constexpr uint32_t kStage = ((kAst + TM * 4 + 1023) / 1024) * 1024;  // + V_I
    static constexpr uint32_t kCol = 4 * 2 * 64 * 4;                    // [quarter][half][64]
    static constexpr uint32_t kBars = 1024;
    static constexpr uint32_t kTotal = 1024 + kB + STAGES_TCS * kStage + kCol + kBars;
};

// Sums 64 values per lane (columns 0..63, one row per lane) over the 32
// lanes: five halving steps across lane bits 16, 8, 4, 2, 1, each sending
// half of the columns a lane holds to its partner and adding the other half
// to the partner's copy, leave in lane l the sums over all 32 rows of the
// columns c and c + 1 in v[0] and v[1], c = 32 b4 + 16 b3 + 8 b2 + 4 b1 +
// 2 b0 (b_k = bit k of l; tcs_colsum_col).
__device__ __forceinline__ void tcs_colsum64(float (&v)[64], int lane) {
#pragma unroll
    for (int w = 64, m = 16; w > 2; w >>= 1, m >>= 1) {
        const bool u = (lane & m) != 0;
        const int hw = w >> 1;
#pragma unroll
        for (int q = 0; q < hw; ++q) {
            const float snd = u ? v[q] : v[q + hw];
            const float kep = u ? v[q + hw] : v[q];
            v[q] = kep + __shfl_xor_sync(0xffffffffu, snd, m);
        }
    }
}

// First of the two columns tcs_colsum64 leaves in lane l (the second is +1).
__device__ __forceinline__ int tcs_colsum_col(int lane) {
    int c = 0;
#pragma unroll
    for (int w = 64, m = 16; w > 2; w >>= 1, m >>= 1)
        if (lane & m) c += w >> 1;
    return c;
}

// Index of the row partials of tile pair (I, J), I <= J.
__host__ __device__ __forceinline__ int64_t tcs_pair(int64_t J, int64_t I) {
    return J * (J + 1) / 2 + I;
}

template <int KCH>
__global__ void __launch_bounds__(SWARPS_TCS * 32, 1)
    kv_tcs_kernel(const __nv_bfloat16* __restrict__ Aop, const __nv_bfloat16* __restrict__ Bop,
                  const float* __restrict__ Vs, const int4* __restrict__ work,
                  float* __restrict__ prow, float* __restrict__ pcol, int* __restrict__ err,
                  uint64_t wait_ns, int stall) {
    using S = TcsSmem<KCH>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;
    uint8_t* sStage = smem + S::kB;
    float* colbuf = reinterpret_cast<float*>(sStage + STAGES_TCS * S::kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sStage + STAGES_TCS * S::kStage + S::kCol);
    uint64_t* full = bars;                       // [STAGES] copies landed
    uint64_t* empty = bars + STAGES_TCS;         // [STAGES] MMAs done + epilogue done with V_I
    uint64_t* tfull = bars + 2 * STAGES_TCS;     // [2] accumulator ready
    uint64_t* tempty = tfull + 2;                // [2] accumulator drained
    uint64_t* bfull = tempty + 2;
    uint64_t* done = bfull + 1;
    uint64_t* never = done + 1;  // test hook: no thread ever arrives here
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wk = work[blockIdx.x];
    const int64_t J = wk.x;
    const int64_t I0 = wk.y;
    const int ntiles = wk.z - wk.y;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES_TCS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1 + SEPI_TCS);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], SEPI_TCS);
        }
        mbar_init(bfull, 1);
        mbar_init(done, 1);
        mbar_init(never, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                su32(tmem_slot)),
            "r"(2 * TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint64_t deadline = gtimer() + wait_ns;
    int fail = 0;
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(bfull, S::kB);
            bulk_g2s(sB, Bop + (size_t)J * KCH * SUB, S::kB, bfull);
            int t = 0;
            for (; t < ntiles; ++t) {
                const int s = t % STAGES_TCS;
                if (!mbar_wait(&empty[s], ((uint32_t)(t / STAGES_TCS) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                const int64_t it = I0 + t;
                uint8_t* st = sStage + (size_t)s * S::kStage;
                mbar_expect_tx(&full[s], S::kAst + TM * 4);
                bulk_g2s(st, Aop + (size_t)it * KCH * SUB, S::kAst, &full[s]);
                bulk_g2s(st + S::kAst, Vs + (size_t)it * TM, TM * 4, &full[s]);
            }
            // the CTA exits only once the copies it issued have landed
            const uint64_t dl2 = gtimer() + 200000000ull;
            for (int q = (t > STAGES_TCS ? t - STAGES_TCS : 0); q < t; ++q)
                (void)mbar_wait(&full[q % STAGES_TCS], (uint32_t)(q / STAGES_TCS) & 1u, dl2);
            (void)mbar_wait(bfull, 0, dl2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // test hook: a wait on a barrier nothing arrives at runs out
            if (stall && !mbar_wait(never, 0, deadline)) fail = 1;
            if (!fail && !mbar_wait(bfull, 0, deadline)) fail = 1;
            fence_after();
            const uint32_t b0 = su32(sB);
            for (int t = 0; t < ntiles && !fail; ++t) {
                const int s = t % STAGES_TCS, b = t & 1;
                if (!mbar_wait(&full[s], (uint32_t)(t / STAGES_TCS) & 1u, deadline) ||
                    !mbar_wait(&tempty[b], ((uint32_t)(t >> 1) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                fence_after();
                const uint32_t a0 = su32(sStage + (size_t)s * S::kStage);
                const uint32_t dt = tmem + (uint32_t)(b * TN);
#pragma unroll
                for (int kc = 0; kc < KCH; ++kc)
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        const uint32_t off = (uint32_t)kc * S::kSub + (uint32_t)kk * 32;
                        mma_bf16(dt, sdesc(a0 + off), sdesc(b0 + off), (kc | kk) ? 1u : 0u);
                    }
                mma_commit(&tfull[b]);
                mma_commit(&empty[s]);
            }
            mma_commit(done);
            if (!mbar_wait(done, 0, gtimer() + kWaitNs)) fail = 1;
        }
    } else {
        // this thread's 64 columns of the resident tile: V_J in registers,
        // column accumulators over the row tiles of the item
        float vj[64], cs[64];
        const float* vjp = Vs + (size_t)J * TN + half * 64;
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            vj[j] = vjp[j];
            cs[j] = 0.f;
        }
        const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % STAGES_TCS, b = t & 1;
            const int64_t it = I0 + t;
            const bool mirror = it < J;  // the diagonal tile gives row sums only
            const bool ok = __all_sync(0xffffffffu,
                                       mbar_wait(&tfull[b], (uint32_t)(t >> 1) & 1u, deadline));
            if (!ok) {
                fail = 1;
                break;
            }
            fence_after();
            const float vi = reinterpret_cast<const float*>(
                sStage + (size_t)s * S::kStage + S::kAst)[row];
            float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ps = 0; ps < 4; ++ps) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
                    "%9, %10, %11, %12, %13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(tbase + (uint32_t)(b * TN + ps * 16)));
                asm volatile("tcgen05.wait::ld.sync.aligned;"
                             : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]),
                               "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]),
                               "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                               "+r"(r[15])
                             :
                             : "memory");
                if (ps == 3) {  // the accumulator goes back to the MMA thread
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float e = ex2(__uint_as_float(r[j]));
                    a[j & 3] = fmaf(e, vj[ps * 16 + j], a[j & 3]);
                    if (mirror) cs[ps * 16 + j] = fmaf(e, vi, cs[ps * 16 + j]);
                }
            }
            // V_I has been read: the stage may be refilled
            fence_proxy_async();
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            prow[(tcs_pair(J, it) * 2 + half) * TM + row] = (a[0] + a[1]) + (a[2] + a[3]);
        }
        // column sums of the item: over the 32 rows of the warp, then the four
        // row quarters (fixed order)
        tcs_colsum64(cs, lane);
        const int c = tcs_colsum_col(lane);
        colbuf[(quarter * 2 + half) * 64 + c] = cs[0];
        colbuf[(quarter * 2 + half) * 64 + c + 1] = cs[1];
    }
    if (fail) atomicExch(&s_fail, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < TN) {
        const int h = threadIdx.x >> 6, c = threadIdx.x & 63;
        const float v = ((colbuf[(0 * 2 + h) * 64 + c] + colbuf[(1 * 2 + h) * 64 + c]) +
                         colbuf[(2 * 2 + h) * 64 + c]) + colbuf[(3 * 2 + h) * 64 + c];
        pcol[(size_t)blockIdx.x * TN + threadIdx.x] = v;
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * TN));
    }
}

// O = noise V + the row partials of the point's tile a (pairs (a, J), J >= a,
// two halves each) + the column partials of the work items of column tile a,
// in FP64, in a fixed order, rounded to FP32.
__global__ void tcs_reduce_kernel(const float* __restrict__ prow, const float* __restrict__ pcol,
                                  const int* __restrict__ col_start,
                                  const int* __restrict__ col_items, int64_t n_t,
                                  const float* __restrict__ V, float noise,
                                  float* __restrict__ O, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t a = i / TM;
    const int r = (int)(i % TM);
    double s = (double)noise * (double)V[i];
    for (int64_t J = a; J < n_t; ++J) {
        const float* p = prow + tcs_pair(J, a) * 2 * TM;
        s += (double)p[r] + (double)p[TM + r];
    }
    for (int e = col_start[a]; e < col_start[a + 1]; ++e)
        s += (double)pcol[(size_t)col_items[e] * TN + r];
    O[i] = (float)s;
}

// V column k as FP32, zero past n (the ring's V_I and the resident V_J).
__global__ void tcs_stage_v_kernel(const float* __restrict__ V, int64_t n, int64_t n_pad,
                                   float* __restrict__ Vs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x)
        Vs[i] = (i < n) ? V[i] : 0.f;
}

template <int KCH>
void launch_tcs(const Ctx& h, const float* Vs, float* prow, float* pcol, cudaStream_t st) {
    using S = TcsSmem<KCH>;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_tcs_kernel<KCH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal));
        attr = true;
    }
    const uint64_t wait_ns = h.opt.wait_limit_ns > 0 ? (uint64_t)h.opt.wait_limit_ns : kWaitNs;
    kv_tcs_kernel<KCH><<<(unsigned)h.tcs_nitems, SWARPS_TCS * 32, S::kTotal, st>>>(
        reinterpret_cast<const __nv_bfloat16*>(h.tcA.p),
        reinterpret_cast<const __nv_bfloat16*>(h.tcB.p), Vs,
        reinterpret_cast<const int4*>(h.tcs_work.p), prow, pcol, h.tc_err.p, wait_ns,
        h.opt.wait_stall ? 1 : 0);
    KPCG_LAUNCHED("kv_tcs_kernel");
}

// Work items for n_t tiles: column tile J takes the row tiles 0..J in runs of
// at most G (G for about eight items per SM, 16..128), launched longest
// first; the items of each column tile are listed (CSR) for the reduction.
void tcs_plan(Ctx& h, int64_t n_t) {
    if (h.tcs_n == h.n) return;
    const double total = (double)n_t * (double)(n_t + 1) / 2.0;
    const int sms = sm_count_tc();
    const int G = (int)std::max(16.0, std::min(128.0, std::ceil(total / (8.0 * sms))));
    std::vector<int4> items;
    for (int64_t J = 0; J < n_t; ++J)
        for (int64_t I = 0; I <= J; I += G)
            items.push_back(make_int4((int)J, (int)I, (int)std::min<int64_t>(I + G, J + 1), 0));
    std::stable_sort(items.begin(), items.end(),
                     [](const int4& a, const int4& b) { return (a.z - a.y) > (b.z - b.y); });
    std::vector<int> cols((size_t)n_t + 1 + items.size(), 0);
    for (const int4& it : items) ++cols[(size_t)it.x + 1];
    for (int64_t J = 0; J < n_t; ++J) cols[(size_t)J + 1] += cols[(size_t)J];
    std::vector<int> fill(cols.begin(), cols.begin() + n_t);
    for (size_t e = 0; e < items.size(); ++e)
        cols[(size_t)n_t + 1 + (size_t)fill[(size_t)items[e].x]++] = (int)e;
    int* w = h.tcs_work.need(items.size() * 4);
    int* c = h.tcs_cols.need(cols.size());
    KPCG_CUDA(cudaMemcpyAsync(w, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                              h.stream));
    KPCG_CUDA(cudaMemcpyAsync(c, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice,
                              h.stream));
    KPCG_CUDA(cudaStreamSynchronize(h.stream));
    h.tcs_nitems = (int)items.size();
    h.tcs_n = h.n;
}

}  // namespace

// Usable while its row partials (n_t (n_t + 1) / 2 tile pairs x 2 halves x 128
// FP32 values) stay within 4 GiB, i.e. up to n ~ 370 000; beyond that the
// one-sided kernel evaluates every entry.
bool kv_tcs_usable(const Ctx& h) {
    const double n_t = (double)((h.n + TM - 1) / TM);
    const double bytes = n_t * (n_t + 1.0) / 2.0 * 2.0 * TM * 4.0;
    return h.n > TM && kv_tc_supported(h.d) && bytes <= 4.0 * 1024 * 1024 * 1024;
}

void kv_tcs_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  float noise) {
    if (h.n <= 0 || c <= 0) return;
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int64_t n_pad = ((n + TM - 1) / TM) * TM;
    const int64_t n_t = n_pad / TM;
    tc_prepare(h);  // the BF16x3 operands of kv_tc.cu (and its error flag)
    const int kch = h.tc_kch;
    tcs_plan(h, n_t);
    float* Vs = h.tcsV.need((size_t)n_pad);
    float* prow = h.tcsRow.need((size_t)tcs_pair(n_t, 0) * 2 * TM);
    float* pcol = h.tcsCol.need((size_t)h.tcs_nitems * TN);
    const int* cols = h.tcs_cols.p;
    for (int k = 0; k < c; ++k) {
        tcs_stage_v_kernel<<<(unsigned)std::min<int64_t>((n_pad + 255) / 256, 2048), 256, 0, st>>>(
            V + (int64_t)k * ldv, n, n_pad, Vs);
        KPCG_LAUNCHED("tcs_stage_v_kernel");
        if (kch == 1)
            launch_tcs<1>(h, Vs, prow, pcol, st);
        else
            launch_tcs<2>(h, Vs, prow, pcol, st);
        tcs_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            prow, pcol, cols, cols + n_t + 1, n_t, V + (int64_t)k * ldv, noise,
            O + (int64_t)k * ldo, n);
        KPCG_LAUNCHED("tcs_reduce_kernel");
    }
}

}  // namespace kpcg
