// Tensor-core K.V for sm_103a: tcgen05 MMA with TMEM accumulators.
//
// O = K V + noise V with K_ij = s^2 exp(-1/2 sum_r (x_ir - x_jr)^2 / l_r^2)
// (Eq. 1), entries rebuilt per 128 x 128 tile and never stored (the matrix-free
// product CG needs, Sec. 2.1).
//
// Exponent on the tensor cores.  With x' = (x - mu) / l * sqrt(log2(e)/2) the
// entry is exp2(a_ij), a_ij = log2(s^2) - |x'_i|^2 - |x'_j|^2 + 2 x'_i.x'_j.
// Every row is split (in FP64) into three BF16 parts x' = h + m + l and
// q = log2(s^2)/2 - |x'|^2 likewise; the augmented rows
//     A_i = [ h  h  m  h  l  m | 1 1 1 | qh qm ql ]
//     B_j = 2[ h  m  h  l  h  m ] | qh qm ql | 1 1 1 ]
// make one BF16 MMA chain (FP32 accumulate) produce a_ij directly: the six
// cross products carry 2 x'_i.x'_j to about 2^-24 relative, which keeps the
// error of K at FP32 level (a two-way TF32 split is twice as large, a single
// BF16 or TF32 rounding is useless against a small noise term).  K-dim is
// 6d + 6, padded to 64 (d <= 9) or 128 (d <= 20).  Padding rows of B carry
// q = -1e30 so their entries vanish.
//
// Data movement.  A prep kernel writes A and B in HBM already in the 128-byte
// swizzled K-major shared-memory layout, one 16 KB block per 128 rows and 64
// columns, so a tile moves with a single bulk copy (cp.async.bulk, TMA engine)
// that completes on an mbarrier.  V tiles move the same way.
//
// Roles (10 warps): warp 0 issues bulk copies into a 4-stage ring, warp 1
// owns TMEM (2 x 128 columns: double-buffered accumulators) and issues the
// MMAs from one thread, warps 2..9 drain TMEM with tcgen05.ld, apply exp2 on
// the MUFU and contract with V in FP32 registers.  Each thread owns one row
// and 64 of the 128 columns of a tile.  Every wait is bounded (globaltimer);
// on expiry the kernel records an error code, drains its own work and frees
// TMEM.  Column ranges of K are split across CTAs and added by a second,
// deterministic kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "batch.cuh"
#include "ctx.cuh"
#include "tcgen05.cuh"

namespace kpcg {
namespace {

constexpr int NSTAGE = 4;
constexpr int NWARPS = 10;
constexpr int NEPI = 8;          // epilogue warps

__device__ __forceinline__ void split3(double v, __nv_bfloat16& h, __nv_bfloat16& m,
                                       __nv_bfloat16& l) {
    h = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(h);
    m = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(m);
    l = __double2bfloat16(r2);
}

// One thread per row: build the augmented A and B rows (see file comment).
__global__ void tc_prep_kernel(const double* __restrict__ xs64, int64_t n, int64_t n_pad, int d,
                               int dp, int kch, double scale, double c0,
                               __nv_bfloat16* __restrict__ Aop, __nv_bfloat16* __restrict__ Bop) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const int kdim = kch * KC;
    const int64_t tile = i / TM;
    const int r = (int)(i % TM);
    uint8_t* abase = reinterpret_cast<uint8_t*>(Aop) + (size_t)tile * kch * SUB * 2;
    uint8_t* bbase = reinterpret_cast<uint8_t*>(Bop) + (size_t)tile * kch * SUB * 2;
    auto put = [&](uint8_t* base, int k, __nv_bfloat16 v) {
        const int kc = k / KC, kk = k % KC;
        *reinterpret_cast<__nv_bfloat16*>(base + (size_t)kc * SUB * 2 + swz_off(r, kk)) = v;
    };
    const __nv_bfloat16 z = __float2bfloat16(0.f), one = __float2bfloat16(1.f);
    for (int k = 0; k < kdim; ++k) {
        put(abase, k, z);
        put(bbase, k, z);
    }
    if (i >= n) {  // padding column of K: exp2(-huge) = 0
        put(bbase, 6 * d, __float2bfloat16(-1e30f));
        return;
    }
    double nrm = 0.0;
    for (int q = 0; q < d; ++q) {
        const double x = xs64[i * dp + q] * scale;
        nrm += x * x;
        __nv_bfloat16 h, m, l;
        split3(x, h, m, l);
        const __nv_bfloat16 h2 = __float2bfloat16(2.f * __bfloat162float(h));
        const __nv_bfloat16 m2 = __float2bfloat16(2.f * __bfloat162float(m));
        const __nv_bfloat16 l2 = __float2bfloat16(2.f * __bfloat162float(l));
        put(abase, 0 * d + q, h);
        put(bbase, 0 * d + q, h2);
        put(abase, 1 * d + q, h);
        put(bbase, 1 * d + q, m2);
        put(abase, 2 * d + q, m);
        put(bbase, 2 * d + q, h2);
        put(abase, 3 * d + q, h);
        put(bbase, 3 * d + q, l2);
        put(abase, 4 * d + q, l);
        put(bbase, 4 * d + q, h2);
        put(abase, 5 * d + q, m);
        put(bbase, 5 * d + q, m2);
    }
    __nv_bfloat16 qh, qm, ql;
    split3(0.5 * c0 - nrm, qh, qm, ql);
    put(abase, 6 * d + 0, one);
    put(abase, 6 * d + 1, one);
    put(abase, 6 * d + 2, one);
    put(bbase, 6 * d + 0, qh);
    put(bbase, 6 * d + 1, qm);
    put(bbase, 6 * d + 2, ql);
    put(abase, 6 * d + 3, qh);
    put(abase, 6 * d + 4, qm);
    put(abase, 6 * d + 5, ql);
    put(bbase, 6 * d + 3, one);
    put(bbase, 6 * d + 4, one);
    put(bbase, 6 * d + 5, one);
}

// ---------------------------------------------------------------------------
// Per-point-exact operands (kv_tcx_apply).  The BF16 x3 split above rounds
// every scaled input to ~2^-24: a per-point perturbation, which moves whole
// rows of K together and, against a small noise term, is amplified by
// K_y^{-1} like ||K|| / sigma^2.  Here each x'/S (S a power of two >= max|x'|)
// is cut into TCX_S slices of 8 bits, x'/S = sum_a s_a 2^(-7-8a) with integer
// s_a in [-128, 128] (exact in BF16), and the exponent, in units of
// 2^-14 S^2,
//     a_ij 2^14 / S^2 = qh_i + qh_j + 2 sum_{a+b<TCX_L} s_a(i).s_b(j) 2^(-8(a+b)),
//     qh_i = (log2(s^2)/2 - |x'_i|^2) 2^14 / S^2,
// is one MMA chain ordered by level k = a + b, each level's terms pre-scaled
// by 2^(-8k) (exact in BF16).  Every level-0 product is an integer below 2^15
// and their sum stays below 2^24, so level 0 accumulates exactly; it already
// holds a_ij to about 2^-8 of |x'|^2, so the later, smaller levels are added
// to an accumulator of the size of a_ij itself, and the FP32 roundings are
// relative to a_ij, independent per entry.  qh_i enters as three BF16 parts
// of its integer part at level 0 (paired with a column of ones) and one
// 8-bit part of its fraction per later level.  The dropped levels (a + b >=
// TCX_L) pair two pseudo-random low slices, an error independent per entry of
// order 2^-40 |x'|^2.
constexpr int TCX_S = 5;  // slices of x'/S
constexpr int TCX_L = 5;  // levels kept
struct TcxLayout {
    int off[TCX_L + 1];  // first column of each level; off[TCX_L] = K
    int d;
};

TcxLayout tcx_layout(int d) {
    TcxLayout L;
    L.d = d;
    int o = 0;
    for (int k = 0; k < TCX_L; ++k) {
        L.off[k] = o;
        const int cols = (k == 0) ? d + 6 : (k + 1) * d + 2;
        o += (cols + 15) / 16 * 16;
    }
    L.off[TCX_L] = o;
    return L;
}

__global__ void tcx_absmax_kernel(const double* __restrict__ xs64, int64_t cnt,
                                  double* __restrict__ out) {
    __shared__ double sh[1024];
    double m = 0.0;
    for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) m = fmax(m, fabs(xs64[e]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void tcx_prep_kernel(const double* __restrict__ xs64, int64_t n, int64_t n_pad, int dp,
                                int kch, double scale, double c0, double invS, double qscale,
                                TcxLayout L, __nv_bfloat16* __restrict__ Aop,
                                __nv_bfloat16* __restrict__ Bop) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const int d = L.d;
    const int kdim = kch * KC;
    const int64_t tile = i / TM;
    const int r = (int)(i % TM);
    uint8_t* abase = reinterpret_cast<uint8_t*>(Aop) + (size_t)tile * kch * SUB * 2;
    uint8_t* bbase = reinterpret_cast<uint8_t*>(Bop) + (size_t)tile * kch * SUB * 2;
    auto put = [&](uint8_t* base, int k, double v) {
        const int kc = k / KC, kk = k % KC;
        *reinterpret_cast<__nv_bfloat16*>(base + (size_t)kc * SUB * 2 + swz_off(r, kk)) =
            __double2bfloat16(v);
    };
    for (int k = 0; k < kdim; ++k) {
        put(abase, k, 0.0);
        put(bbase, k, 0.0);
    }
    if (i >= n) {  // padding column of K: exp2(-huge) = 0
        put(bbase, d + 3, -1e30);
        return;
    }
    double sl[TCX_S][10];
    double nrm = 0.0;
    for (int q = 0; q < d; ++q) {
        const double x = xs64[i * dp + q] * scale;
        nrm += x * x;
        double t = x * invS * 128.0;
        for (int a = 0; a < TCX_S; ++a) {
            const double v = rint(t);
            sl[a][q] = v;
            t = (t - v) * 256.0;
        }
    }
    const double qh = (0.5 * c0 - nrm) * qscale;
    const double I = rint(qh);
    double f = qh - I;
    const double I2 = rint(I / 65536.0);
    const double rem = I - I2 * 65536.0;
    const double I1 = rint(rem / 256.0);
    const double I0 = rem - I1 * 256.0;
    double fr[TCX_L];
    fr[0] = 0.0;
    for (int k = 1; k < TCX_L; ++k) {
        const double t = f * 256.0;
        fr[k] = rint(t);
        f = t - fr[k];
    }
    // level 0
    for (int q = 0; q < d; ++q) {
        put(abase, q, sl[0][q]);
        put(bbase, q, 2.0 * sl[0][q]);
    }
    const double parts[3] = {I2 * 65536.0, I1 * 256.0, I0};
    for (int u = 0; u < 3; ++u) {
        put(abase, d + u, parts[u]);
        put(bbase, d + u, 1.0);
        put(abase, d + 3 + u, 1.0);
        put(bbase, d + 3 + u, parts[u]);
    }
    // levels 1 .. TCX_L-1, pre-scaled by 2^(-8k)
    for (int k = 1; k < TCX_L; ++k) {
        const int base = L.off[k];
        const double sc = ldexp(1.0, -8 * k);
        for (int a = 0; a <= k; ++a) {
            const int b = k - a;
            for (int q = 0; q < d; ++q) {
                put(abase, base + a * d + q, sl[a][q] * sc);
                put(bbase, base + a * d + q, 2.0 * sl[b][q]);
            }
        }
        const int e1 = base + (k + 1) * d;
        put(abase, e1, fr[k] * sc);
        put(bbase, e1, 1.0);
        put(abase, e1 + 1, sc);
        put(bbase, e1 + 1, fr[k]);
    }
}

__global__ void tc_stage_v_kernel(const float* __restrict__ V, int64_t ldv, int64_t n,
                                  int64_t n_pad, float* __restrict__ Vs) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x)
        Vs[i + k * n_pad] = (i < n) ? V[i + k * ldv] : 0.f;
}

template <int KCH, int CB, int VPARTS = 1>
struct TcSmem {
    static constexpr int kNst = KCH >= 3 ? 3 : NSTAGE;          // ring depth (smem budget)
    static constexpr uint32_t kSub = SUB * 2;                    // 16 KB
    static constexpr uint32_t kA = KCH * kSub;                   // A tile
    static constexpr uint32_t kBst = KCH * kSub;                 // B part of a stage
    static constexpr uint32_t kVst = VPARTS * CB * TN * 4;       // V part(s) of a stage
    static constexpr uint32_t kStage = ((kBst + kVst + 1023) / 1024) * 1024;
    static constexpr uint32_t kBars = 1024;
    static constexpr uint32_t kTotal = 1024 /*align slack*/ + kA + kNst * kStage + kBars;
};

// EXACT = 0: the operands of tc_prep_kernel, FP32 contraction, FP32 partials.
// EXACT = 1: the per-point-exact operands of tcx_prep_kernel (nmma MMAs of
// K = 16 per tile, the accumulator times escale is the exp2 argument), row
// sums compensated (TwoSum into an FP32 pair), FP64 partials in part64.
// EXACT = 2: as 1, V given as FP32 pairs (hi in Vs, lo in Vs + nv): each
// product e*v_hi enters the TwoSum, e*v_lo the compensation term.
template <int KCH, int CB, int EXACT>
__global__ void __launch_bounds__(NWARPS * 32, KCH == 1 ? 2 : 1)
    kv_tc_kernel(const __nv_bfloat16* __restrict__ Aop, const __nv_bfloat16* __restrict__ Bop,
                 const float* __restrict__ Vs, int64_t n, int64_t n_pad, int ncols,
                 int tiles_per_split, float* __restrict__ part, int* __restrict__ err,
                 int nmma, float escale, double* __restrict__ part64, uint64_t wait_ns,
                 int stall, int64_t nv) {
    constexpr int VP = (EXACT == 2) ? 2 : 1;
    using S = TcSmem<KCH, CB, VP>;
    constexpr int NST = S::kNst;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sStage = smem + S::kA;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kA + NST * S::kStage);
    uint64_t* full = bars;                  // [NST] bulk copies landed
    uint64_t* empty = bars + NST;           // [NST] MMA done + epilogue done with V
    uint64_t* tfull = bars + 2 * NST;       // [2] accumulator ready
    uint64_t* tempty = bars + 2 * NST + 2;  // [2] accumulator drained
    uint64_t* afull = bars + 2 * NST + 4;
    uint64_t* done = bars + 2 * NST + 5;
    uint64_t* never = bars + 2 * NST + 6;   // test hook: no thread ever arrives here
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 7);
    float* comb = reinterpret_cast<float*>(sStage);    // reused after the loop: [CB][TM]
    float2* comb2 = reinterpret_cast<float2*>(sStage);  // EXACT: [CB][TM] pairs
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rt = blockIdx.x;  // row tile
    const int64_t n_ct = n_pad / TN;
    const int64_t jt0 = (int64_t)blockIdx.y * tiles_per_split;
    const int64_t jt1 = min(n_ct, jt0 + tiles_per_split);
    const int ntiles = (int)max((int64_t)0, jt1 - jt0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1 + NEPI);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], NEPI);
        }
        mbar_init(afull, 1);
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
    float acc[CB], cmp[CB];  // row sums; EXACT: their compensation terms
#pragma unroll
    for (int k = 0; k < CB; ++k) acc[k] = cmp[k] = 0.f;
    const int quarter = warp & 3;         // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;     // epilogue: column half of a tile
    const int row = quarter * 32 + lane;  // epilogue: row of the tile

    if (warp == 0) {
        if (lane == 0) {
            // A tile once, then B + V tiles through the ring
            mbar_expect_tx(afull, S::kA);
            bulk_g2s(sA, Aop + (size_t)rt * KCH * SUB, S::kA, afull);
            int t = 0;
            for (; t < ntiles; ++t) {
                const int s = t % NST;
                if (!mbar_wait(&empty[s], ((uint32_t)(t / NST) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                const int64_t jt = jt0 + t;
                uint8_t* st = sStage + (size_t)s * S::kStage;
                mbar_expect_tx(&full[s], S::kBst + (uint32_t)(VP * ncols) * TN * 4);
                bulk_g2s(st, Bop + (size_t)jt * KCH * SUB, S::kBst, &full[s]);
                for (int vp = 0; vp < VP; ++vp)
                    for (int k = 0; k < ncols; ++k)
                        bulk_g2s(st + S::kBst + (size_t)(vp * CB + k) * TN * 4,
                                 Vs + (size_t)vp * nv + (size_t)k * n_pad + jt * TN, TN * 4,
                                 &full[s]);
            }
            // let the copies this thread issued land before the CTA exits (on
            // the failure path some may still be in flight); own, fresh limit
            const uint64_t dl2 = gtimer() + 200000000ull;
            for (int q = (t > NST ? t - NST : 0); q < t; ++q)
                (void)mbar_wait(&full[q % NST], (uint32_t)(q / NST) & 1u, dl2);
            (void)mbar_wait(afull, 0, dl2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // test hook: a wait on a barrier nothing arrives at runs out
            if (stall && !mbar_wait(never, 0, deadline)) fail = 1;
            if (!fail && !mbar_wait(afull, 0, deadline)) fail = 1;
            fence_after();
            const uint32_t a0 = su32(sA);
            for (int t = 0; t < ntiles && !fail; ++t) {
                const int s = t % NST, b = t & 1;
                if (!mbar_wait(&full[s], (uint32_t)(t / NST) & 1u, deadline) ||
                    !mbar_wait(&tempty[b], ((uint32_t)(t >> 1) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                fence_after();
                const uint32_t b0 = su32(sStage + (size_t)s * S::kStage);
                const uint32_t dt = tmem + (uint32_t)(b * TN);
#pragma unroll
                for (int kc = 0; kc < KCH; ++kc)
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        // the exact operands stop at nmma chunks of K = 16
                        if (EXACT && kc * (KC / 16) + kk >= nmma) continue;
                        const uint32_t off = (uint32_t)kc * S::kSub + (uint32_t)kk * 32;
                        mma_bf16(dt, sdesc(a0 + off), sdesc(b0 + off), (kc | kk) ? 1u : 0u);
                    }
                mma_commit(&tfull[b]);
                mma_commit(&empty[s]);
            }
            // drain: this commit arrives once every MMA issued above has finished
            mma_commit(done);
            if (!mbar_wait(done, 0, gtimer() + kWaitNs)) fail = 1;
        }
    } else {
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % NST, b = t & 1;
            // warp-uniform decision: the TMEM loads below are .sync.aligned
            const bool ok = __all_sync(0xffffffffu,
                                       mbar_wait(&tfull[b], (uint32_t)(t >> 1) & 1u, deadline));
            if (!ok) {
                fail = 1;
                break;
            }
            fence_after();
            const float* vst =
                reinterpret_cast<const float*>(sStage + (size_t)s * S::kStage + S::kBst);
            // this thread's 64 columns in NP passes of W (one TMEM wait per
            // pass; NP = 2 where two CTAs share an SM and registers are short);
            // the accumulator goes back to the MMA thread after the last load
            constexpr int NP = (!EXACT && (CB >= 8 || (KCH == 1 && CB >= 2))) ? 2 : 1;
            constexpr int W = 64 / NP;
            // CH independent accumulation chains per column (latency, not
            // throughput, bounds a single chain at 2 epilogue warps per scheduler)
            constexpr int CH = (CB >= 4) ? 2 : 4;
            const uint32_t taddr =
                tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TN + half * 64);
#pragma unroll
            for (int ps = 0; ps < NP; ++ps) {
                uint32_t r[W];
#pragma unroll
                for (int w = 0; w < W; w += 32) tmem_ld32_nw(taddr + ps * W + w, r + w);
                tmem_wait_ld_bind(r);
#pragma unroll
                for (int w = 32; w < W; w += 32) tmem_bind32(r + w);
                if (ps == NP - 1) {
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
#pragma unroll
                for (int j = 0; j < W; ++j)
                    r[j] = __float_as_uint(
                        ex2(EXACT ? __uint_as_float(r[j]) * escale : __uint_as_float(r[j])));
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const float4* vp =
                        reinterpret_cast<const float4*>(vst + k * TN + half * 64 + ps * W);
                    const float4* vpl = reinterpret_cast<const float4*>(
                        vst + (VP - 1) * CB * TN + k * TN + half * 64 + ps * W);
                    float a[CH], cc[CH];
#pragma unroll
                    for (int u = 0; u < CH; ++u) a[u] = cc[u] = 0.f;
#pragma unroll
                    for (int j4 = 0; j4 < W / 4; ++j4) {
                        const float4 v = vp[j4];
                        const float vv[4] = {v.x, v.y, v.z, v.w};
                        float vl[4] = {0.f, 0.f, 0.f, 0.f};
                        if (EXACT == 2) {
                            const float4 w = vpl[j4];
                            vl[0] = w.x, vl[1] = w.y, vl[2] = w.z, vl[3] = w.w;
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = u % CH;
                            const float e = __uint_as_float(r[4 * j4 + u]);
                            if (EXACT) {  // TwoSum of every product into (a, cc)
                                const float pv = e * vv[u];
                                const float sum = a[q] + pv;
                                const float bp = sum - a[q];
                                cc[q] += (a[q] - (sum - bp)) + (pv - bp);
                                if (EXACT == 2) cc[q] = fmaf(e, vl[u], cc[q]);
                                a[q] = sum;
                            } else {
                                a[q] = fmaf(e, vv[u], a[q]);
                            }
                        }
                    }
                    if (EXACT) {
                        // fold the chains into (acc, cmp) with TwoSum, then Fast2Sum
#pragma unroll
                        for (int u = 0; u < CH; ++u) {
                            const float sum = acc[k] + a[u];
                            const float bp = sum - acc[k];
                            cmp[k] += ((acc[k] - (sum - bp)) + (a[u] - bp)) + cc[u];
                            acc[k] = sum;
                        }
                        const float sum = acc[k] + cmp[k];
                        cmp[k] = cmp[k] - (sum - acc[k]);
                        acc[k] = sum;
                    } else {
                        float t = a[0];
#pragma unroll
                        for (int u = 1; u < CH; ++u) t += a[u];
                        acc[k] += t;
                    }
                }
            }
            fence_proxy_async();
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    // every role ends here
    if (fail) atomicExch(&s_fail, 1);
    fence_before();
    __syncthreads();
    fence_after();
    // add the two column halves of each row (ring memory is free now)
    if (warp >= 2 && half == 1)
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            if (EXACT)
                comb2[k * TM + row] = make_float2(acc[k], cmp[k]);
            else
                comb[k * TM + row] = acc[k];
        }
    __syncthreads();
    if (warp >= 2 && half == 0) {
        const int64_t i = rt * TM + row;
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            if (k >= ncols || i >= n) continue;
            if (EXACT) {
                const float2 o = comb2[k * TM + row];
                part64[((size_t)blockIdx.y * CB + k) * n_pad + i] =
                    ((double)acc[k] + (double)cmp[k]) + ((double)o.x + (double)o.y);
            } else {
                part[((size_t)blockIdx.y * CB + k) * n_pad + i] = acc[k] + comb[k * TM + row];
            }
        }
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * TN));
    }
}

__global__ void tc_reduce_kernel(const float* __restrict__ part, int64_t n_pad, int nsplit,
                                 int cb, int ncols, const float* __restrict__ V, int64_t ldv,
                                 float noise, float* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    float s = noise * V[i + (int64_t)k * ldv];
    for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * cb + k) * n_pad + i];
    O[i + (int64_t)k * ldo] = s;
}


template <int KCH, int CB, int EXACT = 0>
void launch_tc(const Ctx& h, const __nv_bfloat16* A, const __nv_bfloat16* B, const float* Vs,
               int64_t n_pad, int ncols, float* part, int nsplit, int tps, int* err,
               cudaStream_t st, int nmma = 0, float escale = 1.f, double* part64 = nullptr,
               int64_t nv = 0) {
    const uint64_t wait_ns =
        h.opt.wait_limit_ns > 0 ? (uint64_t)h.opt.wait_limit_ns : kWaitNs;
    using S = TcSmem<KCH, CB, EXACT == 2 ? 2 : 1>;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_tc_kernel<KCH, CB, EXACT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal));
        attr = true;
    }
    dim3 grid((unsigned)(n_pad / TM), (unsigned)nsplit);
    kv_tc_kernel<KCH, CB, EXACT><<<grid, NWARPS * 32, S::kTotal, st>>>(
        A, B, Vs, h.n, n_pad, ncols, tps, part, err, nmma, escale, part64, wait_ns,
        h.opt.wait_stall ? 1 : 0, nv);
    KPCG_LAUNCHED(EXACT ? "kv_tcx_kernel" : "kv_tc_kernel");
}

// V (FP64) staged as FP32 pairs: hi at Vs, lo at Vs + nv (column k at k n_pad).
__global__ void tc_stage_v64_kernel(const double* __restrict__ V, int64_t ldv, int64_t n,
                                    int64_t n_pad, float* __restrict__ Vs, int64_t nv) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (i < n) ? V[i + k * ldv] : 0.0;
        const float hi = (float)v;
        Vs[i + k * n_pad] = hi;
        Vs[nv + i + k * n_pad] = (float)(v - (double)hi);
    }
}

// O = noise V + the FP64 partial sums of the exact kernel, in FP64.
__global__ void tcx_reduce64_kernel(const double* __restrict__ part, int64_t n_pad, int nsplit,
                                    int cb, int ncols, const double* __restrict__ V, int64_t ldv,
                                    double noise, double* __restrict__ O, int64_t ldo,
                                    int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    double s = noise * V[i + (int64_t)k * ldv];
    for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * cb + k) * n_pad + i];
    O[i + (int64_t)k * ldo] = s;
}

// O = noise V + the FP64 partial sums of the exact kernel, rounded to FP32.
__global__ void tcx_reduce_kernel(const double* __restrict__ part, int64_t n_pad, int nsplit,
                                  int cb, int ncols, const float* __restrict__ V, int64_t ldv,
                                  float noise, float* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    double s = (double)noise * (double)V[i + (int64_t)k * ldv];
    for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * cb + k) * n_pad + i];
    O[i + (int64_t)k * ldo] = (float)s;
}

}  // namespace

int sm_count_tc() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        if (cached <= 0) cached = 148;
    }
    return cached;
}

bool kv_tc_supported(int d) { return d >= 1 && 6 * d + 6 <= 2 * KC; }


void tc_prepare(Ctx& h) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int64_t n_pad = ((n + TM - 1) / TM) * TM;
    const int kch = (6 * h.d + 6 <= KC) ? 1 : 2;
    if (6 * h.d + 6 > 2 * KC) fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
    if (h.tc_version != h.theta_version || h.tc_kch != kch) {
        h.tcA.need((size_t)n_pad * kch * KC);
        h.tcB.need((size_t)n_pad * kch * KC);
        tc_prep_kernel<<<(unsigned)((n_pad + 127) / 128), 128, 0, st>>>(
            h.xs64.p, n, n_pad, h.d, h.dp, kch, std::sqrt(kLog2e), std::log2(h.s2),
            reinterpret_cast<__nv_bfloat16*>(h.tcA.p), reinterpret_cast<__nv_bfloat16*>(h.tcB.p));
        KPCG_LAUNCHED("tc_prep_kernel");
        h.tc_version = h.theta_version;
        h.tc_kch = kch;
        int* e = h.tc_err.need(1);
        KPCG_CUDA(cudaMemsetAsync(e, 0, sizeof(int), st));
    }
}

void kv_tc_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo, float noise) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int64_t n_pad = ((n + TM - 1) / TM) * TM;
    tc_prepare(h);
    const int kch = h.tc_kch;
    const int n_ct = (int)(n_pad / TN);
    const int n_rt = (int)(n_pad / TM);
    // splits of the column range: about four waves of two CTAs per SM
    int nsplit = std::max(1, std::min(n_ct, (sm_count_tc() * 4 + n_rt - 1) / n_rt));
    const int tps = (n_ct + nsplit - 1) / nsplit;
    nsplit = (n_ct + tps - 1) / tps;
    const int max_cb = 8;
    float* Vs = h.tcV.need((size_t)n_pad * max_cb);
    float* part = h.tcPart.need((size_t)nsplit * max_cb * n_pad);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        tc_stage_v_kernel<<<dim3((unsigned)std::min<int64_t>((n_pad + 255) / 256, 2048),
                                 (unsigned)ncols),
                            256, 0, st>>>(V + (int64_t)k0 * ldv, ldv, n, n_pad, Vs);
        KPCG_LAUNCHED("tc_stage_v_kernel");
        const __nv_bfloat16* A = reinterpret_cast<const __nv_bfloat16*>(h.tcA.p);
        const __nv_bfloat16* B = reinterpret_cast<const __nv_bfloat16*>(h.tcB.p);
#define KPCG_TC_CASE(KCHV, CBV)                                                             \
    if (kch == KCHV && cb == CBV)                                                           \
        launch_tc<KCHV, CBV>(h, A, B, Vs, n_pad, ncols, part, nsplit, tps, h.tc_err.p, st);
        KPCG_TC_CASE(1, 1)
        KPCG_TC_CASE(1, 2)
        KPCG_TC_CASE(1, 4)
        KPCG_TC_CASE(1, 8)
        KPCG_TC_CASE(2, 1)
        KPCG_TC_CASE(2, 2)
        KPCG_TC_CASE(2, 4)
        KPCG_TC_CASE(2, 8)
#undef KPCG_TC_CASE
        tc_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            part, n_pad, nsplit, cb, ncols, V + (int64_t)k0 * ldv, ldv, noise,
            O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("tc_reduce_kernel");
        k0 += ncols;
    }
}

bool kv_tcx_supported(int d) { return d >= 1 && d <= 10; }

static void tcx_prepare(Ctx& h) {
    if (h.tcx_version == h.theta_version) return;
    if (!kv_tcx_supported(h.d)) fail(KPCG_ERR_ARG, "exact tensor-core K.V supports d <= 10");
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int64_t n_pad = ((n + TM - 1) / TM) * TM;
    const TcxLayout L = tcx_layout(h.d);
    const int kch = (L.off[TCX_L] + KC - 1) / KC;
    double* mx = h.tcx_max.need(1);
    tcx_absmax_kernel<<<1, 1024, 0, st>>>(h.xs64.p, n * h.dp, mx);
    KPCG_LAUNCHED("tcx_absmax_kernel");
    double hmax = 0.0;
    KPCG_CUDA(cudaMemcpyAsync(&hmax, mx, sizeof(double), cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    const double scale = std::sqrt(kLog2e);
    const double xmax = hmax * scale;
    double S = 1.0;
    while (S < xmax) S *= 2.0;
    while (S > 2.0 * xmax && S > 1.0 / 1024.0 && xmax > 0.0) S *= 0.5;
    h.tcxA.need((size_t)n_pad * kch * KC);
    h.tcxB.need((size_t)n_pad * kch * KC);
    tcx_prep_kernel<<<(unsigned)((n_pad + 127) / 128), 128, 0, st>>>(
        h.xs64.p, n, n_pad, h.dp, kch, scale, std::log2(h.s2), 1.0 / S, 16384.0 / (S * S), L,
        reinterpret_cast<__nv_bfloat16*>(h.tcxA.p), reinterpret_cast<__nv_bfloat16*>(h.tcxB.p));
    KPCG_LAUNCHED("tcx_prep_kernel");
    h.tcx_kch = kch;
    h.tcx_nmma = L.off[TCX_L] / 16;
    h.tcx_escale = (float)(S * S / 16384.0);
    h.tcx_version = h.theta_version;
    if (!h.tc_err.p) {
        int* e = h.tc_err.need(1);
        KPCG_CUDA(cudaMemsetAsync(e, 0, sizeof(int), st));
    }
}

void kv_tcx_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  float noise) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    if (n <= 0 || c <= 0) return;
    const int64_t n_pad = ((n + TM - 1) / TM) * TM;
    tcx_prepare(h);
    const int kch = h.tcx_kch;
    if (kch != 2 && kch != 3) fail(KPCG_ERR_ARG, "internal: exact operand layout");
    const int n_ct = (int)(n_pad / TN);
    const int n_rt = (int)(n_pad / TM);
    // one CTA per SM (about 200 KB of shared memory each): about four waves
    int nsplit = std::max(1, std::min(n_ct, (sm_count_tc() * 4 + n_rt - 1) / n_rt));
    const int tps = (n_ct + nsplit - 1) / nsplit;
    nsplit = (n_ct + tps - 1) / tps;
    const int max_cb = 8;
    float* Vs = h.tcV.need((size_t)n_pad * max_cb);
    double* part = h.tcxPart.need((size_t)nsplit * max_cb * n_pad);
    const __nv_bfloat16* A = reinterpret_cast<const __nv_bfloat16*>(h.tcxA.p);
    const __nv_bfloat16* B = reinterpret_cast<const __nv_bfloat16*>(h.tcxB.p);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        tc_stage_v_kernel<<<dim3((unsigned)std::min<int64_t>((n_pad + 255) / 256, 2048),
                                 (unsigned)ncols),
                            256, 0, st>>>(V + (int64_t)k0 * ldv, ldv, n, n_pad, Vs);
        KPCG_LAUNCHED("tc_stage_v_kernel");
#define KPCG_TCX_CASE(KCHV, CBV)                                                             \
    if (kch == KCHV && cb == CBV)                                                            \
        launch_tc<KCHV, CBV, 1>(h, A, B, Vs, n_pad, ncols, nullptr, nsplit, tps, h.tc_err.p, st, \
                                h.tcx_nmma, h.tcx_escale, part);
        KPCG_TCX_CASE(2, 1)
        KPCG_TCX_CASE(2, 2)
        KPCG_TCX_CASE(2, 4)
        KPCG_TCX_CASE(2, 8)
        KPCG_TCX_CASE(3, 1)
        KPCG_TCX_CASE(3, 2)
        KPCG_TCX_CASE(3, 4)
        KPCG_TCX_CASE(3, 8)
#undef KPCG_TCX_CASE
        tcx_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            part, n_pad, nsplit, cb, ncols, V + (int64_t)k0 * ldv, ldv, noise,
            O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("tcx_reduce_kernel");
        k0 += ncols;
    }
}

void kv_tcx_apply64(Ctx& h, const double* V, int64_t ldv, int c, double* O, int64_t ldo,
                    double noise) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    if (n <= 0 || c <= 0) return;
    const int64_t n_pad = ((n + TM - 1) / TM) * TM;
    tcx_prepare(h);
    const int kch = h.tcx_kch;
    if (kch != 2 && kch != 3) fail(KPCG_ERR_ARG, "internal: exact operand layout");
    const int n_ct = (int)(n_pad / TN);
    const int n_rt = (int)(n_pad / TM);
    int nsplit = std::max(1, std::min(n_ct, (sm_count_tc() * 4 + n_rt - 1) / n_rt));
    const int tps = (n_ct + nsplit - 1) / nsplit;
    nsplit = (n_ct + tps - 1) / tps;
    const int max_cb = 4;
    const int64_t nv = n_pad * max_cb;
    float* Vs = h.tcV.need((size_t)2 * nv);
    double* part = h.tcxPart.need((size_t)nsplit * max_cb * n_pad);
    const __nv_bfloat16* A = reinterpret_cast<const __nv_bfloat16*>(h.tcxA.p);
    const __nv_bfloat16* B = reinterpret_cast<const __nv_bfloat16*>(h.tcxB.p);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        tc_stage_v64_kernel<<<dim3((unsigned)std::min<int64_t>((n_pad + 255) / 256, 2048),
                                   (unsigned)ncols),
                              256, 0, st>>>(V + (int64_t)k0 * ldv, ldv, n, n_pad, Vs, nv);
        KPCG_LAUNCHED("tc_stage_v64_kernel");
#define KPCG_TCX2_CASE(KCHV, CBV)                                                              \
    if (kch == KCHV && cb == CBV)                                                             \
        launch_tc<KCHV, CBV, 2>(h, A, B, Vs, n_pad, ncols, nullptr, nsplit, tps, h.tc_err.p, st, \
                                h.tcx_nmma, h.tcx_escale, part, nv);
        KPCG_TCX2_CASE(2, 1)
        KPCG_TCX2_CASE(2, 2)
        KPCG_TCX2_CASE(2, 4)
        KPCG_TCX2_CASE(3, 1)
        KPCG_TCX2_CASE(3, 2)
        KPCG_TCX2_CASE(3, 4)
#undef KPCG_TCX2_CASE
        tcx_reduce64_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            part, n_pad, nsplit, cb, ncols, V + (int64_t)k0 * ldv, ldv, noise,
            O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("tcx_reduce64_kernel");
        k0 += ncols;
    }
}

// ------------------------------------------------------------------------
// Batched product over many problems of uneven size: one persistent launch
// walks a flat work list of (problem, row-tile pair, run of column tiles)
// items.  A pair of row tiles shares every column tile: two MMAs per column
// tile into two TMEM accumulators (2 x 2 x 128 columns with double
// buffering), and each epilogue thread owns row r of both tiles, so each value
// of V read from shared memory (a broadcast read, the kernel's bound) serves
// two rows.
// The three roles walk the same items in the same order, so the ring and
// accumulator phases simply continue from one item to the next; the A tile of
// an item is reloaded once the MMAs of the previous item have finished with
// it (aempty).  The K-dim (64 or 128) is per problem.  Each epilogue thread
// writes the partial of its row and column half per item; a second kernel
// adds the items of a row tile in a fixed order.
namespace {

constexpr int kMaxKch = 2;

template <int CB>
struct TcBSmem {
    static constexpr uint32_t kSub = SUB * 2;
    static constexpr uint32_t kA1 = kMaxKch * kSub;  // one row tile of A
    static constexpr uint32_t kA = 2 * kA1;
    static constexpr uint32_t kBst = kMaxKch * kSub;
    static constexpr uint32_t kVst = CB * TN * 4;
    static constexpr uint32_t kStage = ((kBst + kVst + 1023) / 1024) * 1024;
    static constexpr uint32_t kBars = 1024;
    static constexpr uint32_t kTotal = 1024 + kA + NSTAGE * kStage + kBars;
};

__device__ __forceinline__ bool prob_live(const int* __restrict__ active, int p, int cpp) {
    if (!active) return true;
    for (int k = 0; k < cpp; ++k)
        if (active[p * cpp + k]) return true;
    return false;
}

template <int CB>
__global__ void __launch_bounds__(NWARPS * 32, 1)
    kv_tc_batch_kernel(const TcBatchProb* __restrict__ probs,
                       const TcBatchItem* __restrict__ items, int nitems,
                       const float* __restrict__ Vs, int64_t nv, int ncols,
                       const int* __restrict__ active, int cpp, float* __restrict__ part,
                       int* __restrict__ err) {
    using S = TcBSmem<CB>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sStage = smem + S::kA;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kA + NSTAGE * S::kStage);
    uint64_t* full = bars;
    uint64_t* empty = bars + NSTAGE;
    uint64_t* tfull = bars + 2 * NSTAGE;
    uint64_t* tempty = bars + 2 * NSTAGE + 2;
    uint64_t* afull = bars + 2 * NSTAGE + 4;
    uint64_t* aempty = bars + 2 * NSTAGE + 5;
    uint64_t* done = bars + 2 * NSTAGE + 6;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSTAGE + 7);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1 + NEPI);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], NEPI);
        }
        mbar_init(afull, 1);
        mbar_init(aempty, 1);
        mbar_init(done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                su32(tmem_slot)),
            "r"(4 * TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint64_t deadline = gtimer() + kWaitNs;
    int fail = 0;
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t t = 0, u = 0;
            for (int it = blockIdx.x; it < nitems && !fail; it += gridDim.x) {
                const TcBatchItem w = items[it];
                if (!prob_live(active, w.prob, cpp)) continue;
                const TcBatchProb pb = probs[w.prob];
                const uint32_t abytes = (uint32_t)pb.kch * S::kSub;
                if (!mbar_wait(aempty, (u & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                mbar_expect_tx(afull, w.two ? 2 * abytes : abytes);
                bulk_g2s(sA, pb.A + (size_t)w.rt * pb.kch * SUB, abytes, afull);
                if (w.two)
                    bulk_g2s(sA + S::kA1, pb.A + (size_t)(w.rt + 1) * pb.kch * SUB, abytes,
                             afull);
                ++u;
                for (int j = 0; j < w.nt; ++j) {
                    const int s = (int)(t % NSTAGE);
                    if (!mbar_wait(&empty[s], ((t / NSTAGE) & 1u) ^ 1u, deadline)) {
                        fail = 1;
                        break;
                    }
                    const int64_t jt = (int64_t)w.jt0 + j;
                    uint8_t* st = sStage + (size_t)s * S::kStage;
                    mbar_expect_tx(&full[s], abytes + (uint32_t)ncols * TN * 4);
                    bulk_g2s(st, pb.B + (size_t)jt * pb.kch * SUB, abytes, &full[s]);
                    for (int k = 0; k < ncols; ++k)
                        bulk_g2s(st + S::kBst + (size_t)k * TN * 4,
                                 Vs + (size_t)k * nv + pb.voff + jt * TN, TN * 4, &full[s]);
                    ++t;
                }
            }
            // let the copies this thread issued land before the CTA exits
            const uint64_t dl2 = gtimer() + 200000000ull;
            for (uint32_t q = (t > (uint32_t)NSTAGE ? t - NSTAGE : 0u); q < t; ++q)
                (void)mbar_wait(&full[q % NSTAGE], (q / NSTAGE) & 1u, dl2);
            if (u > 0) (void)mbar_wait(afull, (u - 1) & 1u, dl2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t t = 0, u = 0;
            const uint32_t a0 = su32(sA);
            for (int it = blockIdx.x; it < nitems && !fail; it += gridDim.x) {
                const TcBatchItem w = items[it];
                if (!prob_live(active, w.prob, cpp)) continue;
                const int kch = probs[w.prob].kch;
                const int nsub = w.two ? 2 : 1;
                if (!mbar_wait(afull, u & 1u, deadline)) {
                    fail = 1;
                    break;
                }
                ++u;
                fence_after();
                for (int j = 0; j < w.nt; ++j) {
                    const int s = (int)(t % NSTAGE), b = (int)(t & 1u);
                    if (!mbar_wait(&full[s], (t / NSTAGE) & 1u, deadline) ||
                        !mbar_wait(&tempty[b], ((t >> 1) & 1u) ^ 1u, deadline)) {
                        fail = 1;
                        break;
                    }
                    fence_after();
                    const uint32_t b0 = su32(sStage + (size_t)s * S::kStage);
                    for (int sub = 0; sub < nsub; ++sub) {
                        const uint32_t dt = tmem + (uint32_t)(b * 2 * TN + sub * TN);
                        const uint32_t as = a0 + (uint32_t)sub * S::kA1;
                        for (int kc = 0; kc < kch; ++kc)
#pragma unroll
                            for (int kk = 0; kk < KC / 16; ++kk) {
                                const uint32_t off = (uint32_t)kc * S::kSub + (uint32_t)kk * 32;
                                mma_bf16(dt, sdesc(as + off), sdesc(b0 + off),
                                         (kc | kk) ? 1u : 0u);
                            }
                    }
                    mma_commit(&tfull[b]);
                    mma_commit(&empty[s]);
                    ++t;
                }
                if (fail) break;
                mma_commit(aempty);  // the A tile is free once these MMAs finished
            }
            mma_commit(done);
            if (!mbar_wait(done, 0, gtimer() + kWaitNs)) fail = 1;
        }
    } else {
        uint32_t t = 0;
        for (int it = blockIdx.x; it < nitems && !fail; it += gridDim.x) {
            const TcBatchItem w = items[it];
            if (!prob_live(active, w.prob, cpp)) continue;
            const bool two = w.two != 0;  // uniform over the CTA
            float acc[CB], acc2[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) acc[k] = acc2[k] = 0.f;
            for (int j = 0; j < w.nt; ++j) {
                const int s = (int)(t % NSTAGE), b = (int)(t & 1u);
                const bool ok = __all_sync(
                    0xffffffffu, mbar_wait(&tfull[b], (t >> 1) & 1u, deadline));
                if (!ok) {
                    fail = 1;
                    break;
                }
                fence_after();
                const float* vst =
                    reinterpret_cast<const float*>(sStage + (size_t)s * S::kStage + S::kBst);
                const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
                for (int ch = 0; ch < 4; ++ch) {
                    const int col0 = half * 64 + ch * 16;
                    uint32_t r[16];
                    tmem_ld16(trow + (uint32_t)(b * 2 * TN + col0), r);
                    float ev[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) ev[q] = ex2(__uint_as_float(r[q]));
                    // every accumulator runs; those past ncols read stale staging
                    // memory and are never stored (no per-column branch here)
                    if (two) {
                        tmem_ld16(trow + (uint32_t)(b * 2 * TN + TN + col0), r);
                        float ev2[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) ev2[q] = ex2(__uint_as_float(r[q]));
#pragma unroll
                        for (int k = 0; k < CB; ++k) {
                            const float4* vp =
                                reinterpret_cast<const float4*>(vst + k * TN + col0);
                            float a = acc[k], a2 = acc2[k];
#pragma unroll
                            for (int j4 = 0; j4 < 4; ++j4) {
                                const float4 v = vp[j4];
                                a = fmaf(ev[4 * j4 + 0], v.x, a);
                                a2 = fmaf(ev2[4 * j4 + 0], v.x, a2);
                                a = fmaf(ev[4 * j4 + 1], v.y, a);
                                a2 = fmaf(ev2[4 * j4 + 1], v.y, a2);
                                a = fmaf(ev[4 * j4 + 2], v.z, a);
                                a2 = fmaf(ev2[4 * j4 + 2], v.z, a2);
                                a = fmaf(ev[4 * j4 + 3], v.w, a);
                                a2 = fmaf(ev2[4 * j4 + 3], v.w, a2);
                            }
                            acc[k] = a;
                            acc2[k] = a2;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < CB; ++k) {
                            const float4* vp =
                                reinterpret_cast<const float4*>(vst + k * TN + col0);
                            float a = acc[k];
#pragma unroll
                            for (int j4 = 0; j4 < 4; ++j4) {
                                const float4 v = vp[j4];
                                a = fmaf(ev[4 * j4 + 0], v.x, a);
                                a = fmaf(ev[4 * j4 + 1], v.y, a);
                                a = fmaf(ev[4 * j4 + 2], v.z, a);
                                a = fmaf(ev[4 * j4 + 3], v.w, a);
                            }
                            acc[k] = a;
                        }
                    }
                }
                fence_proxy_async();
                fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&tempty[b]);
                    mbar_arrive(&empty[s]);
                }
                ++t;
            }
            if (fail) break;
            // partials [item][sub][half][column][row]
            const int64_t base = (((int64_t)it * 2 + 0) * 2 + half) * CB;
            const int64_t base2 = (((int64_t)it * 2 + 1) * 2 + half) * CB;
#pragma unroll
            for (int k = 0; k < CB; ++k)
                if (k < ncols) {
                    part[(base + k) * TM + row] = acc[k];
                    if (two) part[(base2 + k) * TM + row] = acc2[k];
                }
        }
    }
    if (fail) atomicExch(&s_fail, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(4 * TN));
    }
}

// Vs[k][voff_p + i] = V[i][p*cpp + k0 + k] (zero past n_p).
__global__ void tc_batch_stage_v_kernel(const TcBatchProb* __restrict__ probs,
                                        const float* __restrict__ V, int64_t ldv, int cpp, int k0,
                                        int ncols, int64_t nv, float* __restrict__ Vs) {
    const int p = blockIdx.y;
    const TcBatchProb pb = probs[p];
    for (int k = 0; k < ncols; ++k) {
        const float* v = V + ((int64_t)p * cpp + k0 + k) * ldv;
        float* o = Vs + (int64_t)k * nv + pb.voff;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pb.n_pad;
             i += (int64_t)gridDim.x * blockDim.x)
            o[i] = (i < pb.n) ? v[i] : 0.f;
    }
}

// O[i][p*cpp + k0 + k] = noise_p V + sum over the items of the row-tile pair
// of i in order (both column halves); zero past n_p and for skipped problems.
__global__ void tc_batch_reduce_kernel(const TcBatchProb* __restrict__ probs,
                                       const int32_t* __restrict__ rt_first,
                                       const int32_t* __restrict__ rt_count,
                                       const float* __restrict__ part, int cb, int ncols, int cpp,
                                       int k0, const float* __restrict__ V, int64_t ldv,
                                       float* __restrict__ O, int64_t ldo, int64_t nrows,
                                       const int* __restrict__ active) {
    const int p = blockIdx.y / ncols, k = blockIdx.y % ncols;
    const TcBatchProb pb = probs[p];
    const bool live = prob_live(active, p, cpp);
    const int64_t col = (int64_t)p * cpp + k0 + k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (live && i < pb.n) {
            const int rt = (int)(i / TM), r = (int)(i % TM);
            const int pair = rt >> 1, sub = rt & 1;
            const int f = rt_first[pb.rt_base + pair], cnt = rt_count[pb.rt_base + pair];
            float s = pb.noise * V[col * ldv + i];
            for (int q = 0; q < cnt; ++q) {
                const int64_t base = (((int64_t)(f + q) * 2 + sub) * 2) * cb;
                s += part[(base + k) * TM + r] + part[(base + cb + k) * TM + r];
            }
            v = s;
        }
        O[col * ldo + i] = v;
    }
}

template <int CB>
void launch_tc_batch(TcBatch& b, int ncols, const int* active, int cpp, cudaStream_t st) {
    using S = TcBSmem<CB>;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_tc_batch_kernel<CB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal));
        attr = true;
    }
    const int grid = std::max(1, std::min(b.grid, b.nitems));
    kv_tc_batch_kernel<CB><<<grid, NWARPS * 32, S::kTotal, st>>>(
        b.probs.p, b.items.p, b.nitems, b.Vs.p, b.nv, ncols, active, cpp, b.part.p, b.err.p);
    KPCG_LAUNCHED("kv_tc_batch_kernel");
}

}  // namespace

void tc_batch_plan(TcBatch& b, const std::vector<Ctx*>& subs, const std::vector<float>& noise,
                   int G, int grid, cudaStream_t st, int tcv) {
    if (G < 1) fail(KPCG_ERR_ARG, "tiles per item must be >= 1");
    b.P = (int)subs.size();
    b.G = G;
    b.tcv = tcv ? 1 : 0;
    b.grid = grid > 0 ? grid : sm_count_tc();
    b.hprobs.assign((size_t)b.P, TcBatchProb{});
    std::vector<TcBatchItem> items;
    std::vector<int32_t> first, count;
    int64_t voff = 0;
    int32_t rt_base = 0;
    for (int p = 0; p < b.P; ++p) {
        Ctx& h = *subs[(size_t)p];
        if (b.tcv)
            tcv_prepare(h);  // the same operands, with the dimension check of the tcv path
        else
            tc_prepare(h);
        const int64_t n_pad = ((h.n + TM - 1) / TM) * TM;
        const int n_t = (int)(n_pad / TM);
        TcBatchProb& pb = b.hprobs[(size_t)p];
        pb.A = h.tcA.p;
        pb.B = h.tcB.p;
        pb.voff = voff;
        pb.n = (int32_t)h.n;
        pb.n_pad = (int32_t)n_pad;
        pb.kch = h.tc_kch;
        pb.rt_base = rt_base;
        pb.noise = noise[(size_t)p];
        pb.s2 = (float)h.s2;
        // pairs of row tiles share the V reads of the FP32 contraction; the
        // tensor-core contraction takes one row tile per item
        const int step = b.tcv ? 1 : 2;
        for (int rt = 0; rt < n_t; rt += step) {
            const int two = (!b.tcv && rt + 1 < n_t) ? 1 : 0;
            first.push_back((int32_t)items.size());
            int cnt = 0;
            for (int jt0 = 0; jt0 < n_t; jt0 += G, ++cnt)
                items.push_back(TcBatchItem{p, rt, jt0, std::min(G, n_t - jt0), two, 0});
            count.push_back(cnt);
        }
        voff += n_pad;
        rt_base += (n_t + step - 1) / step;
    }
    b.nv = voff;
    b.nitems = (int)items.size();
    b.probs.need(b.hprobs.size());
    b.items.need(items.size());
    b.rt_first.need(first.size());
    b.rt_count.need(count.size());
    KPCG_CUDA(cudaMemcpyAsync(b.probs.p, b.hprobs.data(), sizeof(TcBatchProb) * b.hprobs.size(),
                              cudaMemcpyHostToDevice, st));
    KPCG_CUDA(cudaMemcpyAsync(b.items.p, items.data(), sizeof(TcBatchItem) * items.size(),
                              cudaMemcpyHostToDevice, st));
    KPCG_CUDA(cudaMemcpyAsync(b.rt_first.p, first.data(), sizeof(int32_t) * first.size(),
                              cudaMemcpyHostToDevice, st));
    KPCG_CUDA(cudaMemcpyAsync(b.rt_count.p, count.data(), sizeof(int32_t) * count.size(),
                              cudaMemcpyHostToDevice, st));
    if (b.tcv) {
        b.Vh.need((size_t)b.nv * 64);
        b.part.need((size_t)b.nitems * 32 * TM);
        b.aux.need((size_t)b.P * 64);
    } else {
        b.Vs.need((size_t)b.nv * 16);
        b.part.need((size_t)b.nitems * 2 * 2 * 16 * TM);
    }
    if (!b.err.p) {
        b.err.need(1);
        KPCG_CUDA(cudaMemsetAsync(b.err.p, 0, sizeof(int), st));
    }
    // the host vectors above are released at return: finish the copies first
    KPCG_CUDA(cudaStreamSynchronize(st));
}

void kv_tc_batch(TcBatch& b, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                 int64_t nrows, const int* active, cudaStream_t st) {
    if (b.P == 0) return;
    if (b.tcv) {
        kv_tcv_batch(b, V, ldv, c, O, ldo, nrows, active, st);
        return;
    }
    int64_t nmax_pad = 0;
    for (const auto& pb : b.hprobs) nmax_pad = std::max<int64_t>(nmax_pad, pb.n_pad);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem > 12 ? 16 : rem > 9 ? 12 : rem == 9 ? 9 : rem > 4 ? 8 : rem > 2 ? 4
                                                                           : rem;
        const int ncols = std::min(cb, rem);
        tc_batch_stage_v_kernel<<<dim3((unsigned)std::min<int64_t>((nmax_pad + 255) / 256, 64),
                                       (unsigned)b.P),
                                  256, 0, st>>>(b.probs.p, V, ldv, c, k0, ncols, b.nv, b.Vs.p);
        KPCG_LAUNCHED("tc_batch_stage_v_kernel");
        switch (cb) {
            case 1: launch_tc_batch<1>(b, ncols, active, c, st); break;
            case 2: launch_tc_batch<2>(b, ncols, active, c, st); break;
            case 4: launch_tc_batch<4>(b, ncols, active, c, st); break;
            case 8: launch_tc_batch<8>(b, ncols, active, c, st); break;
            case 9: launch_tc_batch<9>(b, ncols, active, c, st); break;
            case 12: launch_tc_batch<12>(b, ncols, active, c, st); break;
            default: launch_tc_batch<16>(b, ncols, active, c, st); break;
        }
        tc_batch_reduce_kernel<<<dim3((unsigned)std::min<int64_t>((nrows + 255) / 256, 64),
                                      (unsigned)(b.P * ncols)),
                                 256, 0, st>>>(b.probs.p, b.rt_first.p, b.rt_count.p, b.part.p, cb,
                                               ncols, c, k0, V, ldv, O, ldo, nrows, active);
        KPCG_LAUNCHED("tc_batch_reduce_kernel");
        k0 += ncols;
    }
}

int kv_tc_batch_error(TcBatch& b, cudaStream_t st) {
    if (!b.err.p) return 0;
    int e = 0;
    KPCG_CUDA(cudaMemcpyAsync(&e, b.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    if (e) KPCG_CUDA(cudaMemsetAsync(b.err.p, 0, sizeof(int), st));
    return e;
}

int kv_tc_error(Ctx& h) {
    if (!h.tc_err.p) return 0;
    int e = 0;
    KPCG_CUDA(cudaMemcpyAsync(&e, h.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    KPCG_CUDA(cudaStreamSynchronize(h.stream));
    if (e) KPCG_CUDA(cudaMemsetAsync(h.tc_err.p, 0, sizeof(int), h.stream));
    return e;
}

}  // namespace kpcg
