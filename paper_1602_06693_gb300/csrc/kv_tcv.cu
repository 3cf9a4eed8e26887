// Tensor-core K.V with both contractions on the tensor cores (sm_103a).
//
// O = K V + noise V, K_ij = s^2 exp(-1/2 sum_r (x_ir - x_jr)^2 / l_r^2) (Eq. 1),
// entries rebuilt per 128 x 128 tile and never stored (the matrix-free product
// of Sec. 2.1).
//
// First contraction (the exponent): the BF16x3 augmented operands of kv_tc.cu
// (shared with it); the epilogue scales ex2 of the accumulator by the power of
// two 2^(14 - e_s), 2^e_s > s^2, so E'_ij = K_ij 2^(14 - e_s) < 2^14 (the FP16
// range) exactly.  (Folding the 14 into the exponent instead left the large,
// near-diagonal entries with exponents near 14, whose FP32 accumulation error
// is 14 times coarser and biased.)
//
// Second contraction (E'.V): the epilogue turns each accumulator row into
// E' = hi + lo, two FP16 values (11 + 11 significant bits), and writes them
// back over the accumulator in tensor memory.  A second MMA chain reads them
// as its A operand straight from TMEM (no shared-memory round trip: with
// N = 2c columns the tile would be read from shared memory once per 2c output
// columns, far slower than the ex2 of its entries) against V from shared
// memory.  V is staged per column k as V' = V 2^(14 - e_k), 2^e_k >= max|V_k|,
// split the same way; B rows (2k, 2k+1) = (hi, lo) of column k, so the MMA
// accumulates E'.V'hi and E'.V'lo in adjacent FP32 columns.  Each product
// carries ~2^-21 relative error, independent per entry; the epilogue's work
// per entry (ex2, two FP16 conversions) no longer grows with the number of
// columns, which is what made the FP32-FMA contraction of kv_tc.cu the bound
// from a few columns on.
//
// Roles (10 warps, one CTA per SM): warp 0 bulk-copies the exponent B tile and
// the V tile of each column tile into a ring; warp 1 owns TMEM (two 128-column
// exponent accumulators S, two product accumulators D) and issues from one
// thread the exponent MMAs of tile t into S[t&1], then the E'V MMAs of tile
// t-1 (A = S[(t-1)&1] in TMEM) into D[(t-1)&1]; warps 2..9 load S, apply ex2,
// store the FP16 pairs over S, then read D of the previous tile into FP32 row
// sums.  Each epilogue thread owns one row and one half of the tile (64
// columns of S, NB/2 columns of D).  Every wait is bounded (globaltimer); on
// expiry the kernel records an error code, drains its own work and frees
// TMEM.  Column ranges are split across CTAs and added by a second kernel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "batch.cuh"
#include "ctx.cuh"
#include "tcgen05.cuh"

namespace kpcg {
namespace {

constexpr int VWARPS = 10;
constexpr int VEPI = 8;  // epilogue warps

template <int KCH, int NB>
struct TcvSmem {
    static constexpr uint32_t kSub = SUB * 2;                // 16 KB
    static constexpr uint32_t kA = KCH * kSub;               // exponent A tile
    static constexpr uint32_t kBst = KCH * kSub;             // exponent B tile of a stage
    static constexpr uint32_t kVst = NB * 256;               // V tile: NB rows x 128 FP16
    static constexpr uint32_t kStage = ((kBst + kVst + 1023) / 1024) * 1024;
    static constexpr uint32_t kBars = 1024;
    static constexpr int kNst = (1024 + kA + 4 * kStage + kBars <= 227 * 1024) ? 4 : 3;
    static constexpr uint32_t kTotal = 1024 + kA + kNst * kStage + kBars;
};

// kind::f16 instruction descriptor: FP16 x FP16 -> FP32, K-major A and B,
// M = 128, N = NB (a multiple of 16).
template <int NB>
constexpr uint32_t idesc_f16() {
    return (1u << 4) | ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// D (TMEM) += A (TMEM) B (shared-memory descriptor).
__device__ __forceinline__ void mma_f16_ta(uint32_t dt, uint32_t at, uint64_t bd, uint32_t idesc,
                                           uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], "
        "[%1], %2, %3, p;\n\t}" ::"r"(dt),
        "r"(at), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
        "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
        "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// 8 columns without the wait.
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
// Ties 8 loaded registers to a tcgen05.wait::ld issued before (see tmem_bind32).
__device__ __forceinline__ void tmem_bind8(uint32_t* r) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}

template <int KCH, int NB>
__global__ void __launch_bounds__(VWARPS * 32, 1)
    kv_tcv_kernel(const __nv_bfloat16* __restrict__ Aop, const __nv_bfloat16* __restrict__ Bop,
                  const __half* __restrict__ Vop, int64_t n, int64_t n_pad, int ncols,
                  int tiles_per_split, float* __restrict__ part, int* __restrict__ err,
                  uint64_t wait_ns, int stall, float esc) {
    using S = TcvSmem<KCH, NB>;
    constexpr int NST = S::kNst;
    constexpr int HALF = NB / 2;  // D columns read by each epilogue half
    constexpr int KH = NB / 4;    // output columns of each half
    // D regions: consecutive K-chunks of the E'.V MMAs accumulate into
    // separate TMEM regions, added by the epilogue with round-to-nearest
    // (the tensor core's FP32 accumulation is not round-to-nearest: summed
    // over a whole tile its bias acted on smooth vectors like a per-row
    // scaling of K, 15x the FP32-FMA product's error)
    constexpr int RG = (128 / NB) >= 8 ? 8 : (128 / NB) >= 4 ? 4 : 2;
    constexpr int KPR = 8 / RG;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sStage = smem + S::kA;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kA + NST * S::kStage);
    uint64_t* full = bars;               // [NST] bulk copies landed
    uint64_t* empty = bars + NST;        // [NST] E'V MMAs of the stage's tile done
    uint64_t* tfull = bars + 2 * NST;    // [2] exponent accumulator ready
    uint64_t* sfree = tfull + 2;         // [2] E' of the accumulator consumed
    uint64_t* efull = sfree + 2;         // [2] E' stored over the accumulator
    uint64_t* dfull = efull + 2;         // [2] product accumulator ready
    uint64_t* dempty = dfull + 2;        // [2] product accumulator read
    uint64_t* afull = dempty + 2;
    uint64_t* done = afull + 1;
    uint64_t* never = done + 1;          // test hook: no thread ever arrives here
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rt = blockIdx.x;
    const int64_t n_ct = n_pad / TN;
    const int64_t jt0 = (int64_t)blockIdx.y * tiles_per_split;
    const int64_t jt1 = min(n_ct, jt0 + tiles_per_split);
    const int ntiles = (int)max((int64_t)0, jt1 - jt0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&sfree[b], 1);
            mbar_init(&efull[b], VEPI);
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], VEPI);
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
            "r"(512));
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
    float acc[KH];
#pragma unroll
    for (int k = 0; k < KH; ++k) acc[k] = 0.f;

    if (warp == 0) {
        if (lane == 0) {
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
                mbar_expect_tx(&full[s], S::kBst + S::kVst);
                bulk_g2s(st, Bop + (size_t)jt * KCH * SUB, S::kBst, &full[s]);
                bulk_g2s(st + S::kBst, Vop + (size_t)jt * NB * TN, S::kVst, &full[s]);
            }
            // let the copies issued land before the CTA exits; own, fresh limit
            const uint64_t dl2 = gtimer() + 200000000ull;
            for (int q = (t > NST ? t - NST : 0); q < t; ++q)
                (void)mbar_wait(&full[q % NST], (uint32_t)(q / NST) & 1u, dl2);
            (void)mbar_wait(afull, 0, dl2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            if (stall && !mbar_wait(never, 0, deadline)) fail = 1;
            if (!fail && !mbar_wait(afull, 0, deadline)) fail = 1;
            fence_after();
            const uint32_t a0 = su32(sA);
            // the E'.V MMAs of tile u: A = E' hi (part 0) / lo (part 1) in
            // S[u&1] (half h of the tile's columns at 64 h, hi in its first 32
            // TMEM columns, lo in the next 32), B = the V tile of stage u % NST
            auto mma2 = [&](int u) -> bool {
                const int b = u & 1, s = u % NST;
                if (!mbar_wait(&efull[b], (uint32_t)(u >> 1) & 1u, deadline) ||
                    !mbar_wait(&dempty[b], ((uint32_t)(u >> 1) & 1u) ^ 1u, deadline))
                    return false;
                fence_after();
                const uint32_t vb = su32(sStage + (size_t)s * S::kStage + S::kBst);
                const uint32_t sb = tmem + (uint32_t)(b * TN);
                const uint32_t db = tmem + 256u + (uint32_t)(b * 128);
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int kk = 0; kk < TN / 16; ++kk) {
                        const uint32_t at =
                            sb + (uint32_t)((kk >> 2) * 64 + p * 32 + (kk & 3) * 8);
                        const uint64_t bd =
                            sdesc(vb + (uint32_t)((kk >> 2) * (NB * 128) + (kk & 3) * 32));
                        // K-chunk kk into region kk / KPR of D, each region restarted
                        mma_f16_ta(db + (uint32_t)((kk / KPR) * NB), at, bd, idesc_f16<NB>(),
                                   (p | (kk % KPR)) ? 1u : 0u);
                    }
                mma_commit(&sfree[b]);
                mma_commit(&dfull[b]);
                mma_commit(&empty[s]);
                return true;
            };
            for (int t = 0; t < ntiles && !fail; ++t) {
                const int s = t % NST, b = t & 1;
                if (!mbar_wait(&full[s], (uint32_t)(t / NST) & 1u, deadline) ||
                    !mbar_wait(&sfree[b], ((uint32_t)(t >> 1) & 1u) ^ 1u, deadline)) {
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
                        const uint32_t off = (uint32_t)kc * S::kSub + (uint32_t)kk * 32;
                        mma_bf16(dt, sdesc(a0 + off), sdesc(b0 + off), (kc | kk) ? 1u : 0u);
                    }
                mma_commit(&tfull[b]);
                if (t >= 1 && !mma2(t - 1)) fail = 1;
            }
            if (!fail && ntiles >= 1 && !mma2(ntiles - 1)) fail = 1;
            mma_commit(done);
            if (!mbar_wait(done, 0, gtimer() + kWaitNs)) fail = 1;
        }
    } else {
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        // D of tile u into the row sums (columns 2k, 2k+1: E'.V'hi, E'.V'lo)
        auto readD = [&](int u) -> bool {
            const int b = u & 1;
            const bool ok = __all_sync(0xffffffffu,
                                       mbar_wait(&dfull[b], (uint32_t)(u >> 1) & 1u, deadline));
            if (!ok) return false;
            fence_after();
            uint32_t r[RG][HALF];
#pragma unroll
            for (int g = 0; g < RG; ++g) {
                const uint32_t ta =
                    lane_base + 256u + (uint32_t)(b * 128 + g * NB + half * HALF);
#pragma unroll
                for (int w = 0; w < HALF; w += 8) tmem_ld8_nw(ta + w, &r[g][w]);
            }
            tmem_wait_ld();
#pragma unroll
            for (int g = 0; g < RG; ++g)
#pragma unroll
                for (int w = 0; w < HALF; w += 8) tmem_bind8(&r[g][w]);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[b]);
            // the regions' partials added in FP32 with round-to-nearest
#pragma unroll
            for (int k = 0; k < KH; ++k) {
                float t = 0.f;
#pragma unroll
                for (int g = 0; g < RG; ++g)
                    t += __uint_as_float(r[g][2 * k]) + __uint_as_float(r[g][2 * k + 1]);
                acc[k] += t;
            }
            return true;
        };
        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            const bool ok = __all_sync(0xffffffffu,
                                       mbar_wait(&tfull[b], (uint32_t)(t >> 1) & 1u, deadline));
            if (!ok) {
                fail = 1;
                break;
            }
            fence_after();
            const uint32_t ta = lane_base + (uint32_t)(b * TN + half * 64);
            uint32_t r[64];
            tmem_ld32_nw(ta, r);
            tmem_ld32_nw(ta + 32, r + 32);
            tmem_wait_ld_bind(r);
            tmem_bind32(r + 32);
            uint32_t hp[32], lp[32];
#pragma unroll
            for (int w = 0; w < 32; ++w) {
                const float e0 = ex2(__uint_as_float(r[2 * w])) * esc;
                const float e1 = ex2(__uint_as_float(r[2 * w + 1])) * esc;
                const __half2 h = __floats2half2_rn(e0, e1);  // .x (low half): even column
                const float2 hf = __half22float2(h);
                const __half2 l = __floats2half2_rn(e0 - hf.x, e1 - hf.y);
                hp[w] = *reinterpret_cast<const uint32_t*>(&h);
                lp[w] = *reinterpret_cast<const uint32_t*>(&l);
            }
            tmem_st32(ta, hp);
            tmem_st32(ta + 32, lp);
            tmem_wait_st();
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&efull[b]);
            if (t >= 1 && !readD(t - 1)) {
                fail = 1;
                break;
            }
        }
        if (!fail && ntiles >= 1 && !readD(ntiles - 1)) fail = 1;
    }
    if (fail) atomicExch(&s_fail, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp >= 2) {
        const int64_t i = rt * TM + row;
#pragma unroll
        for (int k = 0; k < KH; ++k) {
            const int kk = half * KH + k;
            if (kk < ncols && i < n) part[((size_t)blockIdx.y * (NB / 2) + kk) * n_pad + i] = acc[k];
        }
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// max |V_k| per column (as the bits of a non-negative float, which order as
// unsigned integers).
__global__ void tcv_colmax_kernel(const float* __restrict__ V, int64_t ldv, int64_t n,
                                  unsigned* __restrict__ mx) {
    const int k = blockIdx.y;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(V[i + (int64_t)k * ldv]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&mx[k], __float_as_uint(m));
}

// V as the B operand of the E'.V MMAs: per 128-row tile, NB rows of 128 FP16
// (row 2k: hi of column k of V' = V 2^(14 - e_k), row 2k + 1: lo), K-major in
// two 64-column sub-tiles with the 128-byte swizzle.  One thread per 16-byte
// chunk.  ex[k] = e_k for the reduction.
__global__ void tcv_stage_v_kernel(const float* __restrict__ V, int64_t ldv, int64_t n,
                                   int64_t n_pad, int nb, int ncols,
                                   const unsigned* __restrict__ mx, __half* __restrict__ Vop,
                                   int* __restrict__ ex) {
    const int64_t total = (n_pad / TN) * nb * 16;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t T = idx / (nb * 16);
    const int rem = (int)(idx - T * nb * 16);
    const int r = rem >> 4, q = rem & 15;
    const int st = q >> 3, c8 = q & 7;
    const int k = r >> 1;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (k < ncols) {
        const float m = __uint_as_float(mx[k]);
        int e = 0;
        if (m > 0.f) (void)frexpf(m, &e);  // m < 2^e
        const float sc = ldexpf(1.f, 14 - e);
        if (T == 0 && (r & 1) == 0 && q == 0) ex[k] = e;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float v2[2];
#pragma unroll
            for (int z = 0; z < 2; ++z) {
                const int64_t j = T * TN + st * 64 + c8 * 8 + 2 * u + z;
                const float v = (j < n) ? V[j + (int64_t)k * ldv] * sc : 0.f;
                const __half hv = __float2half_rn(v);
                v2[z] = (r & 1) ? (v - __half2float(hv)) : __half2float(hv);
            }
            const __half2 p = __floats2half2_rn(v2[0], v2[1]);
            w[u] = *reinterpret_cast<const uint32_t*>(&p);
        }
    }
    uint8_t* dst = reinterpret_cast<uint8_t*>(Vop) + (size_t)T * nb * 256 + (size_t)st * nb * 128 +
                   (size_t)r * 128 + (size_t)((c8 ^ (r & 7)) * 16);
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// O = noise V + 2^(e_k + e_s - 28) (sum of the split partials).
__global__ void tcv_reduce_kernel(const float* __restrict__ part, int64_t n_pad, int nsplit, int cb,
                                  int ncols, const float* __restrict__ V, int64_t ldv, float noise,
                                  const int* __restrict__ ex, int es, float* __restrict__ O,
                                  int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    float s = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * cb + k) * n_pad + i];
    O[i + (int64_t)k * ldo] = fmaf(noise, V[i + (int64_t)k * ldv], ldexpf(s, ex[k] + es - 28));
}

// e_s with s^2 < 2^e_s
int tcv_es(double s2) {
    int e = 0;
    (void)std::frexp(s2, &e);
    return e;
}

template <int KCH, int NB>
void launch_tcv(const Ctx& h, const __nv_bfloat16* A, const __nv_bfloat16* B, const __half* Vop,
                int64_t n_pad, int ncols, float* part, int nsplit, int tps, cudaStream_t st) {
    const uint64_t wait_ns = h.opt.wait_limit_ns > 0 ? (uint64_t)h.opt.wait_limit_ns : kWaitNs;
    using S = TcvSmem<KCH, NB>;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_tcv_kernel<KCH, NB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal));
        attr = true;
    }
    dim3 grid((unsigned)(n_pad / TM), (unsigned)nsplit);
    kv_tcv_kernel<KCH, NB><<<grid, VWARPS * 32, S::kTotal, st>>>(
        A, B, Vop, h.n, n_pad, ncols, tps, part, h.tc_err.p, wait_ns, h.opt.wait_stall ? 1 : 0,
        std::ldexp(1.f, 14 - tcv_es(h.s2)));
    KPCG_LAUNCHED("kv_tcv_kernel");
}

}  // namespace

bool kv_tcv_supported(int d) { return d >= 1 && 6 * d + 6 <= 2 * KC; }

void tcv_prepare(Ctx& h) {
    if (!kv_tcv_supported(h.d)) fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
    tc_prepare(h);  // the operands of kv_tc.cu (and its error flag)
}

void kv_tcv_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  float noise) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    if (n <= 0 || c <= 0) return;
    if (!kv_tcv_supported(h.d)) fail(KPCG_ERR_ARG, "tensor-core K.V supports d <= 20");
    const int64_t n_pad = ((n + TM - 1) / TM) * TM;
    tcv_prepare(h);
    const int kch = h.tc_kch;
    const int n_ct = (int)(n_pad / TN);
    const int n_rt = (int)(n_pad / TM);
    // one CTA per SM: about two waves
    int nsplit = std::max(1, std::min(n_ct, (sm_count_tc() * 2 + n_rt - 1) / n_rt));
    const int tps = (n_ct + nsplit - 1) / nsplit;
    nsplit = (n_ct + tps - 1) / tps;
    constexpr int kMaxCols = 32;
    __half* Vop = reinterpret_cast<__half*>(h.tcvV.need((size_t)n_pad * 2 * kMaxCols));
    float* part = h.tcvPart.need((size_t)nsplit * kMaxCols * n_pad);
    unsigned* mx = reinterpret_cast<unsigned*>(h.tcvAux.need(2 * kMaxCols));
    int* ex = h.tcvAux.p + kMaxCols;
    const __nv_bfloat16* A = reinterpret_cast<const __nv_bfloat16*>(h.tcA.p);
    const __nv_bfloat16* B = reinterpret_cast<const __nv_bfloat16*>(h.tcB.p);
    for (int k0 = 0; k0 < c;) {
        const int ncols = std::min(kMaxCols, c - k0);
        const int nb = ncols <= 8 ? 16 : ncols <= 16 ? 32 : ncols <= 24 ? 48 : 64;
        const float* Vk = V + (int64_t)k0 * ldv;
        KPCG_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned) * ncols, st));
        tcv_colmax_kernel<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 512), (unsigned)ncols),
                            256, 0, st>>>(Vk, ldv, n, mx);
        KPCG_LAUNCHED("tcv_colmax_kernel");
        const int64_t chunks = (n_pad / TN) * nb * 16;
        tcv_stage_v_kernel<<<(unsigned)((chunks + 255) / 256), 256, 0, st>>>(
            Vk, ldv, n, n_pad, nb, ncols, mx, Vop, ex);
        KPCG_LAUNCHED("tcv_stage_v_kernel");
#define KPCG_TCV_CASE(KCHV, NBV)                                                    \
    if (kch == KCHV && nb == NBV)                                                   \
        launch_tcv<KCHV, NBV>(h, A, B, Vop, n_pad, ncols, part, nsplit, tps, st);
        KPCG_TCV_CASE(1, 16)
        KPCG_TCV_CASE(1, 32)
        KPCG_TCV_CASE(1, 48)
        KPCG_TCV_CASE(1, 64)
        KPCG_TCV_CASE(2, 16)
        KPCG_TCV_CASE(2, 32)
        KPCG_TCV_CASE(2, 48)
        KPCG_TCV_CASE(2, 64)
#undef KPCG_TCV_CASE
        tcv_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            part, n_pad, nsplit, nb / 2, ncols, Vk, ldv, noise, ex, tcv_es(h.s2),
            O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("tcv_reduce_kernel");
        k0 += ncols;
    }
}


// ------------------------------------------------------------------------
// Batched product over many problems of uneven size with the contraction on
// the tensor cores: the persistent work-list walk of kv_tc_batch_kernel (items
// of (problem, row tile, run of column tiles), the A tile reloaded once the
// exponent MMAs of the previous item finished with it) around the pipeline of
// kv_tcv_kernel.  Tile counters run on across items, so the deferred E'V MMAs
// and D reads of an item's last tile happen during the next item's first
// tile; each epilogue thread writes its row's partials when it has read the
// last D of an item, and a second kernel adds the items of a row tile.
namespace {

template <int NB>
__global__ void __launch_bounds__(VWARPS * 32, 1)
    kv_tcv_batch_kernel(const TcBatchProb* __restrict__ probs,
                        const TcBatchItem* __restrict__ items, int nitems,
                        const __half* __restrict__ Vop, int ncols, const int* __restrict__ active,
                        int cpp, float* __restrict__ part, int* __restrict__ err,
                        uint64_t wait_ns) {
    using S = TcvSmem<2, NB>;  // room for the larger K-dim
    constexpr int NST = S::kNst;
    constexpr int HALF = NB / 2;
    constexpr int KH = NB / 4;
    constexpr int RG = (128 / NB) >= 8 ? 8 : (128 / NB) >= 4 ? 4 : 2;  // see kv_tcv_kernel
    constexpr int KPR = 8 / RG;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sStage = smem + S::kA;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kA + NST * S::kStage);
    uint64_t* full = bars;
    uint64_t* empty = bars + NST;
    uint64_t* tfull = bars + 2 * NST;
    uint64_t* sfree = tfull + 2;
    uint64_t* efull = sfree + 2;
    uint64_t* dfull = efull + 2;
    uint64_t* dempty = dfull + 2;
    uint64_t* afull = dempty + 2;
    uint64_t* aempty = afull + 1;
    uint64_t* done = aempty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto live = [&](int p) {
        if (!active) return true;
        for (int k = 0; k < cpp; ++k)
            if (active[p * cpp + k]) return true;
        return false;
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&sfree[b], 1);
            mbar_init(&efull[b], VEPI);
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], VEPI);
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
            "r"(512));
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
            uint32_t t = 0, u = 0;
            for (int it = blockIdx.x; it < nitems && !fail; it += gridDim.x) {
                const TcBatchItem w = items[it];
                if (!live(w.prob)) continue;
                const TcBatchProb pb = probs[w.prob];
                const uint32_t abytes = (uint32_t)pb.kch * S::kSub;
                if (!mbar_wait(aempty, (u & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                mbar_expect_tx(afull, abytes);
                bulk_g2s(sA, pb.A + (size_t)w.rt * pb.kch * SUB, abytes, afull);
                ++u;
                for (int j = 0; j < w.nt; ++j) {
                    const int s = (int)(t % NST);
                    if (!mbar_wait(&empty[s], ((t / NST) & 1u) ^ 1u, deadline)) {
                        fail = 1;
                        break;
                    }
                    const int64_t jt = (int64_t)w.jt0 + j;
                    uint8_t* st = sStage + (size_t)s * S::kStage;
                    mbar_expect_tx(&full[s], abytes + S::kVst);
                    bulk_g2s(st, pb.B + (size_t)jt * pb.kch * SUB, abytes, &full[s]);
                    bulk_g2s(st + S::kBst, Vop + (size_t)(pb.voff / TN + jt) * NB * TN, S::kVst,
                             &full[s]);
                    ++t;
                }
            }
            const uint64_t dl2 = gtimer() + 200000000ull;
            for (uint32_t q = (t > (uint32_t)NST ? t - NST : 0u); q < t; ++q)
                (void)mbar_wait(&full[q % NST], (q / NST) & 1u, dl2);
            if (u > 0) (void)mbar_wait(afull, (u - 1) & 1u, dl2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t a0 = su32(sA);
            auto mma2 = [&](uint32_t v) -> bool {
                const int b = (int)(v & 1u), s = (int)(v % NST);
                if (!mbar_wait(&efull[b], (v >> 1) & 1u, deadline) ||
                    !mbar_wait(&dempty[b], ((v >> 1) & 1u) ^ 1u, deadline))
                    return false;
                fence_after();
                const uint32_t vb = su32(sStage + (size_t)s * S::kStage + S::kBst);
                const uint32_t sb = tmem + (uint32_t)(b * TN);
                const uint32_t db = tmem + 256u + (uint32_t)(b * 128);
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int kk = 0; kk < TN / 16; ++kk) {
                        const uint32_t at =
                            sb + (uint32_t)((kk >> 2) * 64 + p * 32 + (kk & 3) * 8);
                        const uint64_t bd =
                            sdesc(vb + (uint32_t)((kk >> 2) * (NB * 128) + (kk & 3) * 32));
                        // K-chunk kk into region kk / KPR of D, each region restarted
                        mma_f16_ta(db + (uint32_t)((kk / KPR) * NB), at, bd, idesc_f16<NB>(),
                                   (p | (kk % KPR)) ? 1u : 0u);
                    }
                mma_commit(&sfree[b]);
                mma_commit(&dfull[b]);
                mma_commit(&empty[s]);
                return true;
            };
            uint32_t t = 0, u = 0;
            for (int it = blockIdx.x; it < nitems && !fail; it += gridDim.x) {
                const TcBatchItem w = items[it];
                if (!live(w.prob)) continue;
                const int kch = probs[w.prob].kch;
                if (!mbar_wait(afull, u & 1u, deadline)) {
                    fail = 1;
                    break;
                }
                ++u;
                fence_after();
                for (int j = 0; j < w.nt; ++j) {
                    const int s = (int)(t % NST), b = (int)(t & 1u);
                    if (!mbar_wait(&full[s], (t / NST) & 1u, deadline) ||
                        !mbar_wait(&sfree[b], ((t >> 1) & 1u) ^ 1u, deadline)) {
                        fail = 1;
                        break;
                    }
                    fence_after();
                    const uint32_t b0 = su32(sStage + (size_t)s * S::kStage);
                    const uint32_t dt = tmem + (uint32_t)(b * TN);
                    for (int kc = 0; kc < kch; ++kc)
#pragma unroll
                        for (int kk = 0; kk < KC / 16; ++kk) {
                            const uint32_t off = (uint32_t)kc * S::kSub + (uint32_t)kk * 32;
                            mma_bf16(dt, sdesc(a0 + off), sdesc(b0 + off), (kc | kk) ? 1u : 0u);
                        }
                    mma_commit(&tfull[b]);
                    if (t >= 1 && !mma2(t - 1)) {
                        fail = 1;
                        break;
                    }
                    ++t;
                }
                if (fail) break;
                mma_commit(aempty);  // the A tile is free once these MMAs finished
            }
            if (!fail && t >= 1 && !mma2(t - 1)) fail = 1;
            mma_commit(done);
            if (!mbar_wait(done, 0, gtimer() + kWaitNs)) fail = 1;
        }
    } else {
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        float acc[KH];
#pragma unroll
        for (int k = 0; k < KH; ++k) acc[k] = 0.f;
        auto readD = [&](uint32_t v) -> bool {
            const int b = (int)(v & 1u);
            const bool ok =
                __all_sync(0xffffffffu, mbar_wait(&dfull[b], (v >> 1) & 1u, deadline));
            if (!ok) return false;
            fence_after();
            uint32_t r[RG][HALF];
#pragma unroll
            for (int g = 0; g < RG; ++g) {
                const uint32_t ta =
                    lane_base + 256u + (uint32_t)(b * 128 + g * NB + half * HALF);
#pragma unroll
                for (int w = 0; w < HALF; w += 8) tmem_ld8_nw(ta + w, &r[g][w]);
            }
            tmem_wait_ld();
#pragma unroll
            for (int g = 0; g < RG; ++g)
#pragma unroll
                for (int w = 0; w < HALF; w += 8) tmem_bind8(&r[g][w]);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[b]);
            // the regions' partials added in FP32 with round-to-nearest
#pragma unroll
            for (int k = 0; k < KH; ++k) {
                float t = 0.f;
#pragma unroll
                for (int g = 0; g < RG; ++g)
                    t += __uint_as_float(r[g][2 * k]) + __uint_as_float(r[g][2 * k + 1]);
                acc[k] += t;
            }
            return true;
        };
        auto flush = [&](int item) {
#pragma unroll
            for (int k = 0; k < KH; ++k) {
                const int kk = half * KH + k;
                if (kk < ncols) part[((int64_t)item * 32 + kk) * TM + row] = acc[k];
                acc[k] = 0.f;
            }
        };
        uint32_t t = 0;
        int prev_item = -1;
        bool prev_last = false;
        for (int it = blockIdx.x; it < nitems && !fail; it += gridDim.x) {
            const TcBatchItem w = items[it];
            if (!live(w.prob)) continue;
            int es_p = 0;
            (void)frexpf(probs[w.prob].s2, &es_p);
            const float esc = ldexpf(1.f, 14 - es_p);  // E' = K 2^(14 - e_s) < 2^14
            for (int j = 0; j < w.nt; ++j) {
                const int b = (int)(t & 1u);
                const bool ok =
                    __all_sync(0xffffffffu, mbar_wait(&tfull[b], (t >> 1) & 1u, deadline));
                if (!ok) {
                    fail = 1;
                    break;
                }
                fence_after();
                const uint32_t ta = lane_base + (uint32_t)(b * TN + half * 64);
                uint32_t r[64];
                tmem_ld32_nw(ta, r);
                tmem_ld32_nw(ta + 32, r + 32);
                tmem_wait_ld_bind(r);
                tmem_bind32(r + 32);
                uint32_t hp[32], lp[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const float e0 = ex2(__uint_as_float(r[2 * q])) * esc;
                    const float e1 = ex2(__uint_as_float(r[2 * q + 1])) * esc;
                    const __half2 h = __floats2half2_rn(e0, e1);
                    const float2 hf = __half22float2(h);
                    const __half2 l = __floats2half2_rn(e0 - hf.x, e1 - hf.y);
                    hp[q] = *reinterpret_cast<const uint32_t*>(&h);
                    lp[q] = *reinterpret_cast<const uint32_t*>(&l);
                }
                tmem_st32(ta, hp);
                tmem_st32(ta + 32, lp);
                tmem_wait_st();
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&efull[b]);
                if (t >= 1) {
                    if (!readD(t - 1)) {
                        fail = 1;
                        break;
                    }
                    if (prev_last) flush(prev_item);
                }
                prev_item = it;
                prev_last = (j == w.nt - 1);
                ++t;
            }
        }
        if (!fail && t >= 1) {
            if (!readD(t - 1))
                fail = 1;
            else
                flush(prev_item);
        }
    }
    if (fail) atomicExch(&s_fail, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// max |V| of column k of problem p (columns p*cpp + k0 + k), as float bits.
__global__ void tcv_batch_colmax_kernel(const TcBatchProb* __restrict__ probs,
                                        const float* __restrict__ V, int64_t ldv, int cpp, int k0,
                                        int ncols, unsigned* __restrict__ mx) {
    const int p = blockIdx.y / ncols, k = blockIdx.y % ncols;
    const TcBatchProb pb = probs[p];
    const float* v = V + ((int64_t)p * cpp + k0 + k) * ldv;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pb.n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(v[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&mx[p * 32 + k], __float_as_uint(m));
}

// The V operand tiles of every problem (layout of tcv_stage_v_kernel, tile
// voff_p / 128 + jt), one thread per 16-byte chunk; ex[p * 32 + k] = e_k.
__global__ void tcv_batch_stage_v_kernel(const TcBatchProb* __restrict__ probs,
                                         const float* __restrict__ V, int64_t ldv, int cpp,
                                         int k0, int nb, int ncols,
                                         const unsigned* __restrict__ mx, __half* __restrict__ Vop,
                                         int* __restrict__ ex) {
    const int p = blockIdx.y;
    const TcBatchProb pb = probs[p];
    const int64_t total = (int64_t)(pb.n_pad / TN) * nb * 16;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t T = idx / (nb * 16);
        const int rem = (int)(idx - T * nb * 16);
        const int r = rem >> 4, q = rem & 15;
        const int st = q >> 3, c8 = q & 7;
        const int k = r >> 1;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (k < ncols) {
            const float m = __uint_as_float(mx[p * 32 + k]);
            int e = 0;
            if (m > 0.f) (void)frexpf(m, &e);
            const float sc = ldexpf(1.f, 14 - e);
            if (T == 0 && (r & 1) == 0 && q == 0) ex[p * 32 + k] = e;
            const float* v = V + ((int64_t)p * cpp + k0 + k) * ldv;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float v2[2];
#pragma unroll
                for (int z = 0; z < 2; ++z) {
                    const int64_t j = T * TN + st * 64 + c8 * 8 + 2 * u + z;
                    const float x = (j < pb.n) ? v[j] * sc : 0.f;
                    const __half hv = __float2half_rn(x);
                    v2[z] = (r & 1) ? (x - __half2float(hv)) : __half2float(hv);
                }
                const __half2 h2 = __floats2half2_rn(v2[0], v2[1]);
                w[u] = *reinterpret_cast<const uint32_t*>(&h2);
            }
        }
        uint8_t* dst = reinterpret_cast<uint8_t*>(Vop) + (size_t)(pb.voff / TN + T) * nb * 256 +
                       (size_t)st * nb * 128 + (size_t)r * 128 + (size_t)((c8 ^ (r & 7)) * 16);
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// O[i][p*cpp + k0 + k] = noise_p V + 2^(e + e_s - 28) (sum over the items of
// the row tile of i, in order); zero past n_p and for skipped problems.
__global__ void tcv_batch_reduce_kernel(const TcBatchProb* __restrict__ probs,
                                        const int32_t* __restrict__ rt_first,
                                        const int32_t* __restrict__ rt_count,
                                        const float* __restrict__ part, int ncols, int cpp, int k0,
                                        const int* __restrict__ ex, const float* __restrict__ V,
                                        int64_t ldv, float* __restrict__ O, int64_t ldo,
                                        int64_t nrows, const int* __restrict__ active) {
    const int p = blockIdx.y / ncols, k = blockIdx.y % ncols;
    const TcBatchProb pb = probs[p];
    bool live = true;
    if (active) {
        live = false;
        for (int q = 0; q < cpp; ++q) live = live || active[p * cpp + q];
    }
    const int64_t col = (int64_t)p * cpp + k0 + k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (live && i < pb.n) {
            const int rt = (int)(i / TM), r = (int)(i % TM);
            const int f = rt_first[pb.rt_base + rt], cnt = rt_count[pb.rt_base + rt];
            float s = 0.f;
            for (int q = 0; q < cnt; ++q) s += part[((int64_t)(f + q) * 32 + k) * TM + r];
            int es_p = 0;
            (void)frexpf(pb.s2, &es_p);
            v = fmaf(pb.noise, V[col * ldv + i], ldexpf(s, ex[p * 32 + k] + es_p - 28));
        }
        O[col * ldo + i] = v;
    }
}

template <int NB>
void launch_tcv_batch(TcBatch& b, int ncols, const int* active, int cpp, cudaStream_t st) {
    using S = TcvSmem<2, NB>;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_tcv_batch_kernel<NB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal));
        attr = true;
    }
    const int grid = std::max(1, std::min(b.grid, b.nitems));
    kv_tcv_batch_kernel<NB><<<grid, VWARPS * 32, S::kTotal, st>>>(
        b.probs.p, b.items.p, b.nitems, reinterpret_cast<const __half*>(b.Vh.p), ncols, active,
        cpp, b.part.p, b.err.p, kWaitNs);
    KPCG_LAUNCHED("kv_tcv_batch_kernel");
}

}  // namespace

void kv_tcv_batch(TcBatch& b, const float* V, int64_t ldv, int c, float* O, int64_t ldo,
                  int64_t nrows, const int* active, cudaStream_t st) {
    if (b.P == 0) return;
    int64_t nmax_pad = 0;
    for (const auto& pb : b.hprobs) nmax_pad = std::max<int64_t>(nmax_pad, pb.n_pad);
    unsigned* mx = reinterpret_cast<unsigned*>(b.aux.p);
    int* ex = b.aux.p + (size_t)b.P * 32;
    __half* Vop = reinterpret_cast<__half*>(b.Vh.p);
    for (int k0 = 0; k0 < c;) {
        const int ncols = std::min(32, c - k0);
        const int nb = ncols <= 8 ? 16 : ncols <= 16 ? 32 : ncols <= 24 ? 48 : 64;
        KPCG_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned) * (size_t)b.P * 32, st));
        tcv_batch_colmax_kernel<<<dim3((unsigned)std::min<int64_t>((nmax_pad + 255) / 256, 64),
                                       (unsigned)(b.P * ncols)),
                                  256, 0, st>>>(b.probs.p, V, ldv, c, k0, ncols, mx);
        KPCG_LAUNCHED("tcv_batch_colmax_kernel");
        const int64_t chunks = (nmax_pad / TN) * nb * 16;
        tcv_batch_stage_v_kernel<<<dim3((unsigned)std::min<int64_t>((chunks + 255) / 256, 1024),
                                        (unsigned)b.P),
                                   256, 0, st>>>(b.probs.p, V, ldv, c, k0, nb, ncols, mx, Vop, ex);
        KPCG_LAUNCHED("tcv_batch_stage_v_kernel");
        switch (nb) {
            case 16: launch_tcv_batch<16>(b, ncols, active, c, st); break;
            case 32: launch_tcv_batch<32>(b, ncols, active, c, st); break;
            case 48: launch_tcv_batch<48>(b, ncols, active, c, st); break;
            default: launch_tcv_batch<64>(b, ncols, active, c, st); break;
        }
        tcv_batch_reduce_kernel<<<dim3((unsigned)std::min<int64_t>((nrows + 255) / 256, 64),
                                       (unsigned)(b.P * ncols)),
                                  256, 0, st>>>(b.probs.p, b.rt_first.p, b.rt_count.p, b.part.p,
                                                ncols, c, k0, ex, V, ldv, O, ldo, nrows, active);
        KPCG_LAUNCHED("tcv_batch_reduce_kernel");
        k0 += ncols;
    }
}

}  // namespace kpcg
