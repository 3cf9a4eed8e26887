// Double-float K.V with the squared distances on the tensor cores (sm_103a).
//
// O = K V + noise V (or B - that) with FP64-class entries K_ij = 2^(a_ij),
// a_ij = log2(s^2) - |x'_i - x'_j|^2 (Eq. 1 in the exp2 scaling of kv_df.cu),
// V and O in FP64, entries rebuilt per tile (the matrix-free product of
// Sec. 2.1).  The double-float kernel of kv_df.cu spends ~130 of its ~185
// FP32 instructions per distinct entry on the exact squared distance; here
// the distance comes from tcgen05 MMAs whose FP32 accumulators are exact
// integers, and the epilogue only combines them, takes the double-float exp2
// and contracts with V.
//
// Slices.  With S a power of two >= max |x'|, x'/S = sum_a s_a 2^(-6-8a),
// a = 0..6, integers |s_0| <= 64 and |s_a| <= 128 (exact in BF16); seven
// slices hold the FP64 value x' to 2^-56 S.  For level k = a + b,
//     Q_k(i) = sum_{a+b=k} sum_r s_a(i,r) s_b(i,r),
//     L_k(i,j) = sum_{a+b=k} sum_r s_a(i,r) s_b(j,r),
//     |x'_i - x'_j|^2 = S^2 sum_k 2^(-12-8k) (Q_k(i) + Q_k(j) - 2 L_k(i,j)).
// Each level is one run of MMA columns: A_i = [s_a(i,r) ..., Q parts, 1 1 1],
// B_j = [2 w_k s_b(j,r) ..., -w_k x3, -w_k Q parts] with w_k = S^2
// 2^(-12-8k) (a power of two, exact in BF16) and Q split into three exact
// BF16 parts.  Every product is exact in FP32 and, for one level, every
// partial sum is an integer multiple of w_k below 2^22 w_k, so a level's
// accumulator holds -w_k (Q_k(i) + Q_k(j) - 2 L_k(i,j)) exactly: levels 0, 1,
// 2 and 3 get one accumulator each, levels 4..6 share a fifth (its FP32
// roundings, ~2^-47 of the exponent, and the dropped levels >= 7, ~2^-45,
// are independent per entry).  No per-point quantity is rounded beyond the
// FP64 x' itself (a per-point rounding of ~2^-48, as a double-float norm would
// carry, limits the residual of the n = 65536 system to ~1e-7).
//
// Tiles of 128 rows x 48 columns; five accumulators x 48 columns x 2 buffers
// = 480 TMEM columns.  Roles (10 warps, one CTA per SM): warp 0 bulk-copies
// the column tile's B operand and V (FP32 pairs) into a ring; warp 1 issues
// the MMAs of a tile from one thread (each level group into its accumulator);
// warps 2..9 read the five accumulators in chunks of 8 columns, add them in
// double-float (TwoSum), add log2(s^2), take Tang's table-driven exp2 and
// accumulate the products with V by TwoSum.  Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "df_arith.cuh"
#include "tcgen05.cuh"

namespace kpcg {
namespace {

constexpr int DNS = 7;      // slices
constexpr int DNG = 5;      // accumulator groups: levels {0}, {1}, {2}, {3}, {4, 5, 6}
constexpr int DTN = 48;     // columns per tile (MMA N)
constexpr int DWARPS = 10;
constexpr int DEPI = 8;
constexpr int DNST = 3;     // ring depth

struct TcdLayout {
    int off[DNG + 1];  // first K column of each group (multiples of 16); off[DNG] = K
    int d;
};

__host__ __device__ inline int tcd_level_cols(int k, int d) {
    // slice pairs (a, k - a) with both below DNS, times d, + 3 Q parts + 3 ones
    const int lo = k - (DNS - 1) > 0 ? k - (DNS - 1) : 0;
    const int hi = k < DNS - 1 ? k : DNS - 1;
    return (hi - lo + 1) * d + 6;
}

TcdLayout tcd_layout(int d) {
    TcdLayout L{};
    L.d = d;
    static const int first[DNG + 1] = {0, 1, 2, 3, 4, 7};
    int off = 0;
    for (int g = 0; g < DNG; ++g) {
        L.off[g] = off;
        int cols = 0;
        for (int k = first[g]; k < first[g + 1]; ++k) cols += tcd_level_cols(k, d);
        off += ((cols + 15) / 16) * 16;
    }
    L.off[DNG] = off;
    return L;
}

__device__ __forceinline__ int tcd_group_first_level(int g) { return g < 4 ? g : 4; }
__device__ __forceinline__ int tcd_group_last_level(int g) { return g < 4 ? g : 6; }

// Byte offset of element (r, k) inside a rows x 64 swizzled K-major sub-tile.
__device__ __forceinline__ uint32_t tcd_swz(int r, int k) {
    return (uint32_t)(r * 128 + (((k >> 3) ^ (r & 7)) * 16) + (k & 7) * 2);
}

// Exact three-part BF16 split of an integer |q| < 2^24.
__device__ __forceinline__ void tcd_split_int(double q, float& p2, float& p1, float& p0) {
    const float h = __bfloat162float(__double2bfloat16(q));
    const double r1 = q - (double)h;
    const float m = __bfloat162float(__double2bfloat16(r1));
    const double r2 = r1 - (double)m;
    p2 = h;
    p1 = m;
    p0 = (float)r2;  // an integer below 2^8: exact in BF16
}

// One thread per point: the A row (tiles of 128 rows) and the B row (tiles of
// btn rows: DTN for kv_tcd_kernel, STN for the symmetric kernel) of point i.
// Padding points: A zero, B with -1e30 in its Q part so that the column's
// entries vanish.
__global__ void tcd_prep_kernel(const double* __restrict__ xs64, int64_t n, int64_t na_pad,
                                int64_t nb_pad, int dp, int kch, double scale, double invS,
                                double S2, TcdLayout L, __nv_bfloat16* __restrict__ Aop,
                                __nv_bfloat16* __restrict__ Bop, int btn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nmax = na_pad > nb_pad ? na_pad : nb_pad;
    if (i >= nmax) return;
    const int d = L.d;
    const int kdim = kch * 64;
    const bool doA = i < na_pad, doB = i < nb_pad;
    uint8_t* abase = reinterpret_cast<uint8_t*>(Aop) + (size_t)(i / 128) * kch * 128 * 128;
    const int ar = (int)(i % 128);
    uint8_t* bbase = reinterpret_cast<uint8_t*>(Bop) + (size_t)(i / btn) * kch * btn * 128;
    const int br = (int)(i % btn);
    auto putA = [&](int k, float v) {
        *reinterpret_cast<__nv_bfloat16*>(abase + (size_t)(k >> 6) * 128 * 128 +
                                          tcd_swz(ar, k & 63)) = __float2bfloat16(v);
    };
    auto putB = [&](int k, float v) {
        *reinterpret_cast<__nv_bfloat16*>(bbase + (size_t)(k >> 6) * btn * 128 +
                                          tcd_swz(br, k & 63)) = __float2bfloat16(v);
    };
    for (int k = 0; k < kdim; ++k) {
        if (doA) putA(k, 0.f);
        if (doB) putB(k, 0.f);
    }
    if (i >= n) {
        if (doB) putB(L.off[0] + d + 3, -1e30f);  // level 0, first Q part of B
        return;
    }
    // slices (exact: every step subtracts a value representable in FP64)
    double s[DNS][16];
    for (int r = 0; r < d; ++r) {
        double v = xs64[i * dp + r] * scale * invS;
        const double a0 = rint(v * 64.0);
        s[0][r] = a0;
        v -= a0 / 64.0;
        for (int a = 1; a < DNS; ++a) {
            const double sc = ldexp(1.0, 6 + 8 * a);
            const double sa = rint(v * sc);
            s[a][r] = sa;
            v -= sa / sc;
        }
    }
    for (int g = 0; g < DNG; ++g) {
        int col = L.off[g];
        for (int k = tcd_group_first_level(g); k <= tcd_group_last_level(g); ++k) {
            const double wk = S2 * ldexp(1.0, -12 - 8 * k);
            const int lo = k - (DNS - 1) > 0 ? k - (DNS - 1) : 0;
            const int hi = k < DNS - 1 ? k : DNS - 1;
            double q = 0.0;
            for (int a = lo; a <= hi; ++a)
                for (int r = 0; r < d; ++r) {
                    if (doA) putA(col, (float)s[a][r]);
                    if (doB) putB(col, (float)(2.0 * wk * s[k - a][r]));
                    q += s[a][r] * s[k - a][r];
                    ++col;
                }
            float q2, q1, q0;
            tcd_split_int(q, q2, q1, q0);
            // A: Q(i) parts against B: -w_k; A: ones against B: -w_k Q(j) parts
            if (doA) {
                putA(col + 0, q2);
                putA(col + 1, q1);
                putA(col + 2, q0);
                putA(col + 3, 1.f);
                putA(col + 4, 1.f);
                putA(col + 5, 1.f);
            }
            if (doB) {
                putB(col + 0, (float)-wk);
                putB(col + 1, (float)-wk);
                putB(col + 2, (float)-wk);
                putB(col + 3, (float)(-wk * q2));
                putB(col + 4, (float)(-wk * q1));
                putB(col + 5, (float)(-wk * q0));
            }
            col += 6;
        }
    }
}


template <int KCH, int CB>
struct TcdSmem {
    static constexpr uint32_t kA = KCH * 128 * 128;       // A tile: 128 rows x 64 K per sub-tile
    static constexpr uint32_t kBst = KCH * DTN * 128;     // B tile: DTN rows
    static constexpr uint32_t kVst = CB * DTN * 8;        // V: CB columns of DTN FP32 pairs
    static constexpr uint32_t kStage = ((kBst + kVst + 1023) / 1024) * 1024;
    static constexpr uint32_t kTab = ((NTAB * 8 + 1023) / 1024) * 1024;
    static constexpr uint32_t kBars = 1024;
    static constexpr uint32_t kTotal = 1024 + kA + DNST * kStage + kTab + kBars;
};

// kind::f16 instruction descriptor: BF16 x BF16 -> FP32, K-major, M = 128, N = DTN.
constexpr uint32_t kIdescD =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(DTN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint64_t sdesc_d(uint32_t saddr) { return sdesc(saddr); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <int KCH, int CB>
__global__ void __launch_bounds__(DWARPS * 32, 1)
    kv_tcd_kernel(const __nv_bfloat16* __restrict__ Aop, const __nv_bfloat16* __restrict__ Bop,
                  const float2* __restrict__ Vs, int64_t nb_pad, int64_t n, int ncols,
                  int tiles_per_split, TcdLayout L, float c0h, float c0l,
                  const float2* __restrict__ gtab, double* __restrict__ part,
                  int64_t na_pad, int* __restrict__ err, uint64_t wait_ns) {
    using S = TcdSmem<KCH, CB>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sStage = smem + S::kA;
    float2* tab = reinterpret_cast<float2*>(sStage + DNST * S::kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sStage + DNST * S::kStage + S::kTab);
    uint64_t* full = bars;               // [DNST]
    uint64_t* empty = bars + DNST;       // [DNST] MMAs done + epilogue done with V
    uint64_t* tfull = bars + 2 * DNST;   // [2]
    uint64_t* tempty = tfull + 2;        // [2]
    uint64_t* afull = tempty + 2;
    uint64_t* done = afull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    float2* comb = reinterpret_cast<float2*>(sStage);  // after the loop: [CB][128]
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rt = blockIdx.x;
    const int64_t n_ct = nb_pad / DTN;
    const int64_t jt0 = (int64_t)blockIdx.y * tiles_per_split;
    const int64_t jt1 = min(n_ct, jt0 + tiles_per_split);
    const int ntiles = (int)max((int64_t)0, jt1 - jt0);

    for (int e = threadIdx.x; e < NTAB; e += blockDim.x) tab[e] = gtab[e];
    if (threadIdx.x == 0) {
        for (int s = 0; s < DNST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1 + DEPI);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], DEPI);
        }
        mbar_init(afull, 1);
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
    float Sk[CB], Ck[CB];  // row sums (double-float)
#pragma unroll
    for (int k = 0; k < CB; ++k) Sk[k] = Ck[k] = 0.f;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(afull, S::kA);
            bulk_g2s(sA, Aop + (size_t)rt * KCH * 128 * 64, S::kA, afull);
            int t = 0;
            for (; t < ntiles; ++t) {
                const int s = t % DNST;
                if (!mbar_wait(&empty[s], ((uint32_t)(t / DNST) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                const int64_t jt = jt0 + t;
                uint8_t* st = sStage + (size_t)s * S::kStage;
                mbar_expect_tx(&full[s], S::kBst + (uint32_t)ncols * DTN * 8);
                bulk_g2s(st, Bop + (size_t)jt * KCH * DTN * 64, S::kBst, &full[s]);
                for (int k = 0; k < ncols; ++k)
                    bulk_g2s(st + S::kBst + (size_t)k * DTN * 8, Vs + (size_t)k * nb_pad + jt * DTN,
                             DTN * 8, &full[s]);
            }
            const uint64_t dl2 = gtimer() + 200000000ull;
            for (int q = (t > DNST ? t - DNST : 0); q < t; ++q)
                (void)mbar_wait(&full[q % DNST], (uint32_t)(q / DNST) & 1u, dl2);
            (void)mbar_wait(afull, 0, dl2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            if (!mbar_wait(afull, 0, deadline)) fail = 1;
            fence_after();
            const uint32_t a0 = su32(sA);
            for (int t = 0; t < ntiles && !fail; ++t) {
                const int s = t % DNST, b = t & 1;
                if (!mbar_wait(&full[s], (uint32_t)(t / DNST) & 1u, deadline) ||
                    !mbar_wait(&tempty[b], ((uint32_t)(t >> 1) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                fence_after();
                const uint32_t b0 = su32(sStage + (size_t)s * S::kStage);
                for (int g = 0; g < DNG; ++g) {
                    const uint32_t dt = tmem + (uint32_t)(b * DNG * DTN + g * DTN);
                    for (int c16 = L.off[g] >> 4; c16 < (L.off[g + 1] >> 4); ++c16) {
                        const uint32_t aoff = (uint32_t)(c16 >> 2) * 128 * 128 + (uint32_t)(c16 & 3) * 32;
                        const uint32_t boff = (uint32_t)(c16 >> 2) * DTN * 128 + (uint32_t)(c16 & 3) * 32;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                            "l"(sdesc_d(a0 + aoff)), "l"(sdesc_d(b0 + boff)), "r"(kIdescD),
                            "r"((uint32_t)(c16 != (L.off[g] >> 4))));
                    }
                }
                mma_commit(&tfull[b]);
                mma_commit(&empty[s]);
            }
            mma_commit(done);
            if (!mbar_wait(done, 0, gtimer() + kWaitNs)) fail = 1;
        }
    } else {
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % DNST, b = t & 1;
            const bool ok = __all_sync(0xffffffffu,
                                       mbar_wait(&tfull[b], (uint32_t)(t >> 1) & 1u, deadline));
            if (!ok) {
                fail = 1;
                break;
            }
            fence_after();
            const float2* vst =
                reinterpret_cast<const float2*>(sStage + (size_t)s * S::kStage + S::kBst);
            // this half's DTN / 2 = 24 columns in three chunks of 8
#pragma unroll 1
            for (int ch = 0; ch < 3; ++ch) {
                const int col0 = half * (DTN / 2) + ch * 8;
                uint32_t r[DNG][8];
#pragma unroll
                for (int g = 0; g < DNG; ++g) {
                    const uint32_t ta = lane_base + (uint32_t)(b * DNG * DTN + g * DTN + col0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                        : "=r"(r[g][0]), "=r"(r[g][1]), "=r"(r[g][2]), "=r"(r[g][3]), "=r"(r[g][4]),
                          "=r"(r[g][5]), "=r"(r[g][6]), "=r"(r[g][7])
                        : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int g = 0; g < DNG; ++g)
                    asm volatile(""
                                 : "+r"(r[g][0]), "+r"(r[g][1]), "+r"(r[g][2]), "+r"(r[g][3]),
                                   "+r"(r[g][4]), "+r"(r[g][5]), "+r"(r[g][6]), "+r"(r[g][7])
                                 :
                                 : "memory");
                if (ch == 2) {  // the accumulator goes back to the MMA thread
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    // exponent = log2(s^2) + acc0 + acc1 + acc2 + acc3 + acc4 in double-float:
                    // acc0..acc3 exact, so TwoSum pairs (0, 1) and (2, 3), acc4 into a tail
                    float h, l, u, v;
                    two_sum(__uint_as_float(r[0][q]), __uint_as_float(r[1][q]), h, l);
                    two_sum(__uint_as_float(r[2][q]), __uint_as_float(r[3][q]), u, v);
                    v += __uint_as_float(r[4][q]);
                    float s1, e1;
                    two_sum(h, u, s1, e1);
                    e1 += l + v;
                    float ah, al;
                    two_sum(c0h, s1, ah, al);
                    al += e1 + c0l;
                    const DF e = df_exp2(ah, al, tab);
                    const int jc = col0 + q;
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        const float2 vv = vst[k * DTN + jc];
                        const float P = e.h * vv.x;
                        float Pe = fmaf(e.h, vv.x, -P);
                        Pe = fmaf(e.h, vv.y, Pe);
                        Pe = fmaf(e.l, vv.x, Pe);
                        df_acc(Sk[k], Ck[k], P, Pe);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) df_renorm(Sk[k], Ck[k]);
            fence_proxy_async();
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    if (fail) atomicExch(&s_fail, 1);
    fence_before();
    __syncthreads();
    fence_after();
    // the two column halves of each row (ring memory is free now)
    if (warp >= 2 && half == 1)
#pragma unroll
        for (int k = 0; k < CB; ++k) comb[k * 128 + row] = make_float2(Sk[k], Ck[k]);
    __syncthreads();
    if (warp >= 2 && half == 0) {
        const int64_t i = rt * 128 + row;
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            if (k >= ncols || i >= n) continue;
            const float2 o = comb[k * 128 + row];
            part[((size_t)blockIdx.y * CB + k) * na_pad + i] =
                ((double)Sk[k] + (double)Ck[k]) + ((double)o.x + (double)o.y);
        }
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// V (FP64) as FP32 pairs, column k at k * nb_pad, zero past n.
__global__ void tcd_stage_v_kernel(const double* __restrict__ V, int64_t ldv, int64_t n,
                                   int64_t nb_pad, float2* __restrict__ Vs) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (i < n) ? V[i + (int64_t)k * ldv] : 0.0;
        const float hi = (float)v;
        Vs[i + (int64_t)k * nb_pad] = make_float2(hi, (float)(v - (double)hi));
    }
}

// O = noise V + sum of the split partials (or B minus that), in FP64.
__global__ void tcd_reduce_kernel(const double* __restrict__ part, int64_t na_pad, int nsplit,
                                  int cb, int ncols, const double* __restrict__ V, int64_t ldv,
                                  double noise, const double* __restrict__ B, int64_t ldb,
                                  double* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    double s = noise * V[i + (int64_t)k * ldv];
    for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * cb + k) * na_pad + i];
    O[i + (int64_t)k * ldo] = B ? (B[i + (int64_t)k * ldb] - s) : s;
}

__global__ void tcd_absmax_kernel(const double* __restrict__ xs64, int64_t cnt,
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

// ---------------------------------------------------------------------------
// Symmetric variant.  K is symmetric, so one evaluation per unordered pair of
// points suffices.  Work item (I, J0, J1) pairs row tile I (128 rows, the A
// operand) with column tiles J0..J1-1 of STN = 32 columns.  Column tiles
// inside row block I (J = 4I..4I+3) are evaluated in full and give row sums
// only; tiles right of it (J >= 4I + 4) give the row sums K_IJ V_J and, from
// the same entries, the column sums K_IJ^T V_I.  Every pair of points in
// different row blocks is thus evaluated once, by the lower block's items.
// Sixteen epilogue warps (four row quarters, the TMEM lanes each may read,
// times four groups of 8 columns) keep four warps per scheduler to hide the
// latency of the double-float chains.  A column sum is reduced over the 32
// rows of a warp by a butterfly that halves the columns a lane holds at each
// step (18 shuffles for 8 columns), then over the four row quarters through
// shared memory behind a bounded mbarrier wait, and leaves as one FP64
// partial per (column tile, row tile); a second kernel adds, for every row,
// its row partials and the column partials of all row tiles below it, in a
// fixed order.
constexpr int STN = 32;   // columns per tile of the symmetric kernel (MMA N)
constexpr int SNST = 3;   // ring depth

template <int KCH, int CB>
struct TcdsSmem {
    static constexpr uint32_t kA = KCH * 128 * 128;
    static constexpr uint32_t kBst = KCH * STN * 128;
    static constexpr uint32_t kVst = CB * STN * 8;
    static constexpr uint32_t kStage = ((kBst + kVst + 1023) / 1024) * 1024;
    static constexpr uint32_t kTab = NTAB1K * 8;
    // [set][buf][half][quarter][k][16] float2
    static constexpr uint32_t kCol = 2 * 2 * 2 * 4 * CB * 16 * 8;
    static constexpr uint32_t kBars = 1024;
    static constexpr uint32_t kTotal = 1024 + kA + SNST * kStage + kTab + kCol + kBars;
};

constexpr uint32_t kIdescS =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(STN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr int SEPI = 16;          // epilogue warps: two sets of 4 row quarters x 2 column halves
constexpr int SSET = 8;           // warps per set; set s takes the tiles t = s mod 2
constexpr int SWARPS = 2 + SEPI;  // + the producer and the MMA issuer

// (h, l) += (bh, bl) for double-float values: TwoSum on the high parts.
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
    const float s = h + bh;
    const float bb = s - h;
    const float e = (h - (s - bb)) + (bh - bb);
    h = s;
    l = l + bl + e;
}

// Sums eight double-float values per lane (columns 0..7, one row per lane)
// over the 32 lanes.  While a lane holds w > 1 columns, it sends half of
// them to its partner across the next lane bit (16, 8, 4) and adds the
// other half to the partner's copy; the remaining bits (2, 1) are plain
// reductions.  On return lane l holds the sum over all 32 rows of column
// 4 b4 + 2 b3 + b2 (b_k = bit k of l), in (oh, ol).
__device__ __forceinline__ void df_colsum8(float (&ph)[8], float (&pl)[8], int lane, float& oh,
                                           float& ol) {
#pragma unroll
    for (int w = 8, m = 16; w > 1; w >>= 1, m >>= 1) {
        const bool u = (lane & m) != 0;
        const int hw = w >> 1;
#pragma unroll
        for (int q = 0; q < hw; ++q) {
            const float sh = u ? ph[q] : ph[q + hw], sl = u ? pl[q] : pl[q + hw];
            float kh = u ? ph[q + hw] : ph[q], kl = u ? pl[q + hw] : pl[q];
            const float rh = __shfl_xor_sync(0xffffffffu, sh, m);
            const float rl = __shfl_xor_sync(0xffffffffu, sl, m);
            df_add(kh, kl, rh, rl);
            ph[q] = kh;
            pl[q] = kl;
        }
    }
    oh = ph[0];
    ol = pl[0];
#pragma unroll
    for (int m = 2; m >= 1; m >>= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, oh, m);
        const float rl = __shfl_xor_sync(0xffffffffu, ol, m);
        df_add(oh, ol, rh, rl);
    }
}

// Index of the column partial of (column tile J, row tile I), I < J / 4: the
// pairs are numbered by J, then I.
__host__ __device__ __forceinline__ int64_t tcds_pair(int64_t J, int64_t I) {
    const int64_t u = J >> 2, v = J & 3;
    return 2 * u * (u - 1) + v * u + I;
}

template <int KCH, int CB>
__global__ void __launch_bounds__(SWARPS * 32, 1)
    kv_tcds_kernel(const __nv_bfloat16* __restrict__ Aop, const __nv_bfloat16* __restrict__ Bop,
                   const float2* __restrict__ Vs, int64_t n_pad, int ncols,
                   const int4* __restrict__ work, TcdLayout L, float c0h, float c0l,
                   const float2* __restrict__ gtab, double* __restrict__ prow,
                   double* __restrict__ pcol, int* __restrict__ err, uint64_t wait_ns) {
    using S = TcdsSmem<KCH, CB>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sStage = smem + S::kA;
    float2* tab = reinterpret_cast<float2*>(sStage + SNST * S::kStage);
    float2* colbuf = reinterpret_cast<float2*>(sStage + SNST * S::kStage + S::kTab);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sStage + SNST * S::kStage + S::kTab + S::kCol);
    uint64_t* full = bars;               // [SNST]
    uint64_t* empty = bars + SNST;       // [SNST] MMAs done + epilogue done with V
    uint64_t* tfull = bars + 2 * SNST;   // [2]
    uint64_t* tempty = tfull + 2;        // [2]
    uint64_t* cfull = tempty + 2;        // [set][buf][half] column partials written
    uint64_t* afull = cfull + 8;
    uint64_t* done = afull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    float2* comb = reinterpret_cast<float2*>(sStage);  // after the loop: [CB][4][128]
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wk = work[blockIdx.x];
    const int64_t I = wk.x;
    const int64_t J0 = wk.y;
    const int ntiles = wk.z - wk.y;

    for (int e = threadIdx.x; e < NTAB1K; e += blockDim.x) tab[e] = gtab[e];
    if (threadIdx.x == 0) {
        for (int s = 0; s < SNST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1 + SSET);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], SSET);
        }
        for (int b = 0; b < 8; ++b) mbar_init(&cfull[b], 128);
        mbar_init(afull, 1);
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
    const int quarter = warp & 3;             // TMEM lanes (rows) 32 quarter .. +31
    const int eset = (warp - 2) >> 3;         // tiles t with t mod 2 == eset, TMEM buffer eset
    const int half = ((warp - 2) >> 2) & 1;   // columns 16 half .. +15 of each tile
    const int row = quarter * 32 + lane;
    float Sk[CB], Ck[CB];  // row sums (double-float)
#pragma unroll
    for (int k = 0; k < CB; ++k) Sk[k] = Ck[k] = 0.f;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(afull, S::kA);
            bulk_g2s(sA, Aop + (size_t)I * KCH * 128 * 64, S::kA, afull);
            int t = 0;
            for (; t < ntiles; ++t) {
                const int s = t % SNST;
                if (!mbar_wait(&empty[s], ((uint32_t)(t / SNST) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                const int64_t jt = J0 + t;
                uint8_t* st = sStage + (size_t)s * S::kStage;
                mbar_expect_tx(&full[s], S::kBst + (uint32_t)ncols * STN * 8);
                bulk_g2s(st, Bop + (size_t)jt * KCH * STN * 64, S::kBst, &full[s]);
                for (int k = 0; k < ncols; ++k)
                    bulk_g2s(st + S::kBst + (size_t)k * STN * 8, Vs + (size_t)k * n_pad + jt * STN,
                             STN * 8, &full[s]);
            }
            // the CTA exits only once the copies it issued have landed
            const uint64_t dl2 = gtimer() + 200000000ull;
            for (int q = (t > SNST ? t - SNST : 0); q < t; ++q)
                (void)mbar_wait(&full[q % SNST], (uint32_t)(q / SNST) & 1u, dl2);
            (void)mbar_wait(afull, 0, dl2);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            if (!mbar_wait(afull, 0, deadline)) fail = 1;
            fence_after();
            const uint32_t a0 = su32(sA);
            for (int t = 0; t < ntiles && !fail; ++t) {
                const int s = t % SNST, b = t & 1;
                if (!mbar_wait(&full[s], (uint32_t)(t / SNST) & 1u, deadline) ||
                    !mbar_wait(&tempty[b], ((uint32_t)(t >> 1) & 1u) ^ 1u, deadline)) {
                    fail = 1;
                    break;
                }
                fence_after();
                const uint32_t b0 = su32(sStage + (size_t)s * S::kStage);
                for (int g = 0; g < DNG; ++g) {
                    const uint32_t dt = tmem + (uint32_t)(b * DNG * STN + g * STN);
                    for (int c16 = L.off[g] >> 4; c16 < (L.off[g + 1] >> 4); ++c16) {
                        const uint32_t aoff = (uint32_t)(c16 >> 2) * 128 * 128 + (uint32_t)(c16 & 3) * 32;
                        const uint32_t boff = (uint32_t)(c16 >> 2) * STN * 128 + (uint32_t)(c16 & 3) * 32;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                            "l"(sdesc_d(a0 + aoff)), "l"(sdesc_d(b0 + boff)), "r"(kIdescS),
                            "r"((uint32_t)(c16 != (L.off[g] >> 4))));
                    }
                }
                mma_commit(&tfull[b]);
                mma_commit(&empty[s]);
            }
            mma_commit(done);
            if (!mbar_wait(done, 0, gtimer() + kWaitNs)) fail = 1;
        }
    } else {
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        float2 vi[CB];  // this row's V, for the column sums
#pragma unroll
        for (int k = 0; k < CB; ++k)
            vi[k] = (k < ncols) ? Vs[(size_t)k * n_pad + (size_t)I * 128 + row] : make_float2(0.f, 0.f);
        int mt = 0;  // this set's mirrored tiles so far: the column-partial buffer and its phase
        for (int t = eset; t < ntiles; t += 2) {
            const int s = t % SNST, b = t & 1;
            const int64_t jt = J0 + t;
            const bool mirror = jt >= 4 * I + 4;
            const bool ok = __all_sync(0xffffffffu,
                                       mbar_wait(&tfull[b], (uint32_t)(t >> 1) & 1u, deadline));
            if (!ok) {
                fail = 1;
                break;
            }
            fence_after();
            const float2* vst =
                reinterpret_cast<const float2*>(sStage + (size_t)s * S::kStage + S::kBst);
            const int cbuf = mt & 1;
            float2* mine = colbuf + (size_t)(((eset * 2 + cbuf) * 2 + half) * 4 + quarter) * CB * 16;
#pragma unroll 1
            for (int ch = 0; ch < 2; ++ch) {
                const int col0 = half * (STN / 2) + ch * 8;
                uint32_t r[DNG][8];
#pragma unroll
                for (int g = 0; g < DNG; ++g) {
                    const uint32_t ta = lane_base + (uint32_t)(b * DNG * STN + g * STN + col0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                        : "=r"(r[g][0]), "=r"(r[g][1]), "=r"(r[g][2]), "=r"(r[g][3]), "=r"(r[g][4]),
                          "=r"(r[g][5]), "=r"(r[g][6]), "=r"(r[g][7])
                        : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int g = 0; g < DNG; ++g)
                    asm volatile(""
                                 : "+r"(r[g][0]), "+r"(r[g][1]), "+r"(r[g][2]), "+r"(r[g][3]),
                                   "+r"(r[g][4]), "+r"(r[g][5]), "+r"(r[g][6]), "+r"(r[g][7])
                                 :
                                 : "memory");
                if (ch == 1) {  // the accumulator goes back to the MMA thread
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
                float eh[8], el[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    // exponent = log2(s^2) + acc0 + .. + acc4 in double-float, as kv_tcd_kernel
                    float h, l, u, v;
                    two_sum(__uint_as_float(r[0][q]), __uint_as_float(r[1][q]), h, l);
                    two_sum(__uint_as_float(r[2][q]), __uint_as_float(r[3][q]), u, v);
                    v += __uint_as_float(r[4][q]);
                    float s1, e1;
                    two_sum(h, u, s1, e1);
                    e1 += l + v;
                    float ah, al;
                    two_sum(c0h, s1, ah, al);
                    al += e1 + c0l;
                    const DF e = df_exp2_1k(ah, al, tab);
                    eh[q] = e.h;
                    el[q] = e.l;
                }
#pragma unroll
                for (int k = 0; k < CB; ++k) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float2 vv = vst[k * STN + col0 + q];
                        const float P = eh[q] * vv.x;
                        float Pe = fmaf(eh[q], vv.x, -P);
                        Pe = fmaf(eh[q], vv.y, Pe);
                        Pe = fmaf(el[q], vv.x, Pe);
                        df_acc(Sk[k], Ck[k], P, Pe);
                    }
                }
                if (mirror) {
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        float ph[8], pl[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            ph[q] = eh[q] * vi[k].x;
                            float Pe = fmaf(eh[q], vi[k].x, -ph[q]);
                            Pe = fmaf(eh[q], vi[k].y, Pe);
                            pl[q] = fmaf(el[q], vi[k].x, Pe);
                        }
                        float oh, ol;
                        df_colsum8(ph, pl, lane, oh, ol);
                        if ((lane & 3) == 0) {
                            const int cq = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 +
                                           ((lane >> 2) & 1);
                            mine[k * 16 + ch * 8 + cq] = make_float2(oh, ol);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) df_renorm(Sk[k], Ck[k]);
            fence_proxy_async();
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (mirror) {
                // the four row quarters of this half: their column partials are
                // in shared memory once all 128 threads arrived
                uint64_t* cb = &cfull[(eset * 2 + cbuf) * 2 + half];
                mbar_arrive(cb);
                if (!__all_sync(0xffffffffu, mbar_wait(cb, (uint32_t)(mt >> 1) & 1u, deadline))) {
                    fail = 1;
                    break;
                }
                const float2* base =
                    colbuf + (size_t)((eset * 2 + cbuf) * 2 + half) * 4 * CB * 16;
                const int64_t pair = tcds_pair(jt, I);
                for (int idx = quarter * 32 + lane; idx < CB * 16; idx += 128) {
                    const int k = idx >> 4, col = idx & 15;
                    float h = base[k * 16 + col].x, l = base[k * 16 + col].y;
#pragma unroll
                    for (int q = 1; q < 4; ++q) {
                        const float2 w = base[(q * CB + k) * 16 + col];
                        df_add(h, l, w.x, w.y);
                    }
                    if (k < ncols)
                        pcol[((size_t)pair * CB + k) * STN + half * 16 + col] =
                            (double)h + (double)l;
                }
                ++mt;
            }
        }
    }
    if (fail) atomicExch(&s_fail, 1);
    fence_before();
    __syncthreads();
    fence_after();
    // the four partial row sums of each row (two sets x two column halves;
    // ring memory is free now), added in a fixed order
    const int part = eset * 2 + half;
    if (warp >= 2 && part > 0)
#pragma unroll
        for (int k = 0; k < CB; ++k) comb[(k * 4 + part) * 128 + row] = make_float2(Sk[k], Ck[k]);
    __syncthreads();
    if (warp >= 2 && part == 0) {
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            if (k >= ncols) continue;
            double acc = (double)Sk[k] + (double)Ck[k];
#pragma unroll
            for (int g = 1; g < 4; ++g) {
                const float2 o = comb[(k * 4 + g) * 128 + row];
                acc += (double)o.x + (double)o.y;
            }
            prow[((size_t)blockIdx.x * CB + k) * 128 + row] = acc;
        }
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// O = noise V + this row's partials (its row tile's items, then the column
// partials of every row tile below it), or B minus that, in FP64 and in a
// fixed order.
__global__ void tcds_reduce_kernel(const double* __restrict__ prow, const double* __restrict__ pcol,
                                   const int* __restrict__ row_start, const int* __restrict__ row_items,
                                   int cb, int ncols, const double* __restrict__ V, int64_t ldv,
                                   double noise, const double* __restrict__ B, int64_t ldb,
                                   double* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    const int64_t a = i >> 7;
    double s = noise * V[i + (int64_t)k * ldv];
    for (int e = row_start[a]; e < row_start[a + 1]; ++e)
        s += prow[((size_t)row_items[e] * cb + k) * 128 + (i & 127)];
    const int64_t base = tcds_pair(i >> 5, 0);
    const int c = (int)(i & 31);
#pragma unroll 4
    for (int64_t ip = 0; ip < a; ++ip) s += pcol[((size_t)(base + ip) * cb + k) * STN + c];
    O[i + (int64_t)k * ldo] = B ? (B[i + (int64_t)k * ldb] - s) : s;
}

template <int KCH, int CB>
void launch_tcd(const Ctx& h, const TcdLayout& L, const float2* Vs, int64_t na_pad,
                int64_t nb_pad, int ncols, double* part, int nsplit, int tps, cudaStream_t st) {
    using S = TcdSmem<KCH, CB>;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_tcd_kernel<KCH, CB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal));
        attr = true;
    }
    const uint64_t wait_ns = h.opt.wait_limit_ns > 0 ? (uint64_t)h.opt.wait_limit_ns : kWaitNs;
    dim3 grid((unsigned)(na_pad / 128), (unsigned)nsplit);
    kv_tcd_kernel<KCH, CB><<<grid, DWARPS * 32, S::kTotal, st>>>(
        reinterpret_cast<const __nv_bfloat16*>(h.tcdA.p),
        reinterpret_cast<const __nv_bfloat16*>(h.tcdB.p), Vs, nb_pad, h.n, ncols, tps, L, h.df_c0h,
        h.df_c0l, reinterpret_cast<const float2*>(h.df_tab.p), part, na_pad, h.tc_err.p, wait_ns);
    KPCG_LAUNCHED("kv_tcd_kernel");
}

template <int KCH>
void launch_tcd_cb(int cb, const Ctx& h, const TcdLayout& L, const float2* Vs, int64_t na_pad,
                   int64_t nb_pad, int ncols, double* part, int nsplit, int tps, cudaStream_t st) {
    if (cb == 1)
        launch_tcd<KCH, 1>(h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st);
    else if (cb == 2)
        launch_tcd<KCH, 2>(h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st);
    else
        launch_tcd<KCH, 4>(h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st);
}

}  // namespace

bool kv_tcd_supported(const Ctx& h) { return h.d >= 1 && h.d <= 10; }

namespace {

template <int KCH, int CB>
void launch_tcds(const Ctx& h, const TcdLayout& L, const float2* Vs, int64_t n_pad, int ncols,
                 double* prow, double* pcol, cudaStream_t st) {
    using S = TcdsSmem<KCH, CB>;
    static bool attr = false;
    if (!attr) {
        KPCG_CUDA(cudaFuncSetAttribute(kv_tcds_kernel<KCH, CB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal));
        attr = true;
    }
    const uint64_t wait_ns = h.opt.wait_limit_ns > 0 ? (uint64_t)h.opt.wait_limit_ns : kWaitNs;
    kv_tcds_kernel<KCH, CB><<<(unsigned)h.tcds_nitems, SWARPS * 32, S::kTotal, st>>>(
        reinterpret_cast<const __nv_bfloat16*>(h.tcdA.p),
        reinterpret_cast<const __nv_bfloat16*>(h.tcdBs.p), Vs, n_pad, ncols,
        reinterpret_cast<const int4*>(h.tcds_work.p), L, h.df_c0h, h.df_c0l,
        reinterpret_cast<const float2*>(h.df_tab1k.p), prow, pcol, h.tc_err.p, wait_ns);
    KPCG_LAUNCHED("kv_tcds_kernel");
}

template <int KCH>
void launch_tcds_cb(int cb, const Ctx& h, const TcdLayout& L, const float2* Vs, int64_t n_pad,
                    int ncols, double* prow, double* pcol, cudaStream_t st) {
    if (cb == 1)
        launch_tcds<KCH, 1>(h, L, Vs, n_pad, ncols, prow, pcol, st);
    else if (cb == 2)
        launch_tcds<KCH, 2>(h, L, Vs, n_pad, ncols, prow, pcol, st);
    else
        launch_tcds<KCH, 4>(h, L, Vs, n_pad, ncols, prow, pcol, st);
}

// Sliced operands of the handle's current theta: A in tiles of 128 rows, B in
// tiles of btn rows (into Bbuf), rebuilt when theta changed since `version`.
void tcd_operands(Ctx& h, const TcdLayout& L, int kch, int64_t na_pad, int64_t nb_pad, int btn,
                  DevBuf<uint16_t>& Bbuf, int& version) {
    if (version == h.theta_version) return;
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    double* mx = h.tcd_max.need(1);
    tcd_absmax_kernel<<<1, 1024, 0, st>>>(h.xs64.p, n * h.dp, mx);
    KPCG_LAUNCHED("tcd_absmax_kernel");
    double hmax = 0.0;
    KPCG_CUDA(cudaMemcpyAsync(&hmax, mx, sizeof(double), cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    const double scale = std::sqrt(kLog2e);
    const double xmax = hmax * scale;
    double S = 1.0;
    while (S < xmax) S *= 2.0;
    while (S > 2.0 * xmax && S > 1.0 / 1024.0 && xmax > 0.0) S *= 0.5;
    h.tcdA.need((size_t)na_pad * kch * 64);
    Bbuf.need((size_t)nb_pad * kch * 64);
    const int64_t nmax = std::max(na_pad, nb_pad);
    tcd_prep_kernel<<<(unsigned)((nmax + 127) / 128), 128, 0, st>>>(
        h.xs64.p, n, na_pad, nb_pad, h.dp, kch, scale, 1.0 / S, S * S, L,
        reinterpret_cast<__nv_bfloat16*>(h.tcdA.p), reinterpret_cast<__nv_bfloat16*>(Bbuf.p), btn);
    KPCG_LAUNCHED("tcd_prep_kernel");
    version = h.theta_version;
}

// Work items of the symmetric kernel for n_rt row tiles: row tile I walks the
// column tiles 4I..4 n_rt - 1 in runs of at most G, G chosen for at least
// eight items per SM; the items are launched longest first, and the row
// partials of each row tile are listed (CSR) for the reduction.
void tcds_plan(Ctx& h, int64_t n_rt) {
    if (h.tcds_n == h.n) return;
    const int64_t n_ct = 4 * n_rt;
    const double total = (double)n_rt * (double)n_ct - 2.0 * (double)n_rt * (double)(n_rt - 1);
    const int sms = sm_count_tc();
    const int G = (int)std::max(16.0, std::min(64.0, std::ceil(total / (8.0 * sms))));
    std::vector<int4> items;
    for (int64_t I = 0; I < n_rt; ++I)
        for (int64_t J = 4 * I; J < n_ct; J += G)
            items.push_back(make_int4((int)I, (int)J, (int)std::min<int64_t>(J + G, n_ct), 0));
    std::stable_sort(items.begin(), items.end(),
                     [](const int4& a, const int4& b) { return (a.z - a.y) > (b.z - b.y); });
    std::vector<int> rows((size_t)n_rt + 1 + items.size(), 0);
    for (const int4& it : items) ++rows[(size_t)it.x + 1];
    for (int64_t I = 0; I < n_rt; ++I) rows[(size_t)I + 1] += rows[(size_t)I];
    std::vector<int> fill(rows.begin(), rows.begin() + n_rt);
    for (size_t e = 0; e < items.size(); ++e)
        rows[(size_t)n_rt + 1 + (size_t)fill[(size_t)items[e].x]++] = (int)e;
    int* w = h.tcds_work.need(items.size() * 4);
    int* r = h.tcds_rows.need(rows.size());
    KPCG_CUDA(cudaMemcpyAsync(w, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                              h.stream));
    KPCG_CUDA(cudaMemcpyAsync(r, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice,
                              h.stream));
    KPCG_CUDA(cudaStreamSynchronize(h.stream));
    h.tcds_nitems = (int)items.size();
    h.tcds_n = h.n;
}

// The product on symmetric tile pairs (kv_tcds_kernel + tcds_reduce_kernel).
void kv_tcd_sym(Ctx& h, const TcdLayout& L, int kch, const double* V, int64_t ldv, int c,
                const double* B, int64_t ldb, double* O, int64_t ldo, double noise) {
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const int64_t n_pad = ((n + 127) / 128) * 128;
    const int64_t n_rt = n_pad / 128;
    tcd_operands(h, L, kch, n_pad, n_pad, STN, h.tcdBs, h.tcds_version);
    tcds_plan(h, n_rt);
    const int cbmax = c >= 4 ? 4 : c >= 2 ? 2 : 1;
    const int64_t npairs = tcds_pair(4 * n_rt, 0);
    float2* Vs = h.tcdV.need((size_t)n_pad * 4);
    double* prow = h.tcdsRow.need((size_t)h.tcds_nitems * cbmax * 128);
    double* pcol = h.tcdsCol.need((size_t)std::max<int64_t>(npairs, 1) * cbmax * STN);
    const int* rows = h.tcds_rows.p;
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        const double* Vk = V + (int64_t)k0 * ldv;
        tcd_stage_v_kernel<<<dim3((unsigned)std::min<int64_t>((n_pad + 255) / 256, 2048),
                                  (unsigned)ncols),
                             256, 0, st>>>(Vk, ldv, n, n_pad, Vs);
        KPCG_LAUNCHED("tcd_stage_v_kernel");
        switch (kch) {
            case 2: launch_tcds_cb<2>(cb, h, L, Vs, n_pad, ncols, prow, pcol, st); break;
            case 3: launch_tcds_cb<3>(cb, h, L, Vs, n_pad, ncols, prow, pcol, st); break;
            case 4: launch_tcds_cb<4>(cb, h, L, Vs, n_pad, ncols, prow, pcol, st); break;
            case 5: launch_tcds_cb<5>(cb, h, L, Vs, n_pad, ncols, prow, pcol, st); break;
            default: launch_tcds_cb<6>(cb, h, L, Vs, n_pad, ncols, prow, pcol, st); break;
        }
        tcds_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            prow, pcol, rows, rows + n_rt + 1, cb, ncols, Vk, ldv, noise,
            B ? B + (int64_t)k0 * ldb : nullptr, ldb, O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("tcds_reduce_kernel");
        k0 += ncols;
    }
}

}  // namespace

void kv_tcd(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb, double* O,
            int64_t ldo, double noise) {
    if (h.n <= 0 || c <= 0) return;
    if (!kv_tcd_supported(h)) fail(KPCG_ERR_ARG, "internal: tensor-core double-float K.V needs d <= 10");
    cudaStream_t st = h.stream;
    df_prepare(h);  // exp2 table, log2(s^2) as a double-float pair
    if (!h.tc_err.p) {
        int* e = h.tc_err.need(1);
        KPCG_CUDA(cudaMemsetAsync(e, 0, sizeof(int), st));
    }
    const int64_t n = h.n;
    const TcdLayout L = tcd_layout(h.d);
    const int kch = (L.off[DNG] + 63) / 64;
    if (kch < 2 || kch > 6) fail(KPCG_ERR_ARG, "internal: sliced operand layout");
    // one evaluation per pair of points once there is more than one row tile,
    // while its column partials (2 n_t (n_t - 1) tile pairs x up to 4 columns
    // x 32 FP64 values) stay within 4 GiB; beyond that (n above ~185 000 for
    // four columns, ~370 000 for one) the one-sided kernel evaluates every entry
    const int64_t n_rt_sym = (n + 127) / 128;
    const double sym_bytes = 2.0 * (double)n_rt_sym * (double)(n_rt_sym - 1) *
                             (double)(c >= 4 ? 4 : c >= 2 ? 2 : 1) * STN * 8.0;
    if (h.tcd_symmetric && n > 128 && sym_bytes <= 4.0 * 1024 * 1024 * 1024) {
        kv_tcd_sym(h, L, kch, V, ldv, c, B, ldb, O, ldo, noise);
        return;
    }
    const int64_t na_pad = ((n + 127) / 128) * 128;
    const int64_t nb_pad = ((n + DTN - 1) / DTN) * DTN;
    tcd_operands(h, L, kch, na_pad, nb_pad, DTN, h.tcdB, h.tcd_version);
    // splits of the column range: the CTA count (one per SM) closest above a
    // whole number of waves, with at least 8 column tiles per CTA
    const int n_rt = (int)(na_pad / 128);
    const int n_ct = (int)(nb_pad / DTN);
    const int sms = sm_count_tc();
    int nsplit = 1;
    double best = 1e30;
    for (int ns = 1; ns <= 16; ++ns) {
        const int tps = (n_ct + ns - 1) / ns;
        if (ns > 1 && tps < 8) break;
        const double ctas = (double)n_rt * ((n_ct + tps - 1) / tps);
        const double waves = std::ceil(ctas / sms);
        const double cost = (double)tps * waves;  // time ~ waves x tiles per CTA
        if (cost < best - 1e-9) {
            best = cost;
            nsplit = ns;
        }
    }
    const int tps = (n_ct + nsplit - 1) / nsplit;
    nsplit = (n_ct + tps - 1) / tps;
    constexpr int kMaxCb = 4;
    float2* Vs = h.tcdV.need((size_t)nb_pad * kMaxCb);
    double* part = h.tcdPart.need((size_t)nsplit * kMaxCb * na_pad);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        const double* Vk = V + (int64_t)k0 * ldv;
        tcd_stage_v_kernel<<<dim3((unsigned)std::min<int64_t>((nb_pad + 255) / 256, 2048),
                                  (unsigned)ncols),
                             256, 0, st>>>(Vk, ldv, n, nb_pad, Vs);
        KPCG_LAUNCHED("tcd_stage_v_kernel");
        switch (kch) {
            case 2: launch_tcd_cb<2>(cb, h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st); break;
            case 3: launch_tcd_cb<3>(cb, h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st); break;
            case 4: launch_tcd_cb<4>(cb, h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st); break;
            case 5: launch_tcd_cb<5>(cb, h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st); break;
            default: launch_tcd_cb<6>(cb, h, L, Vs, na_pad, nb_pad, ncols, part, nsplit, tps, st); break;
        }
        tcd_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            part, na_pad, nsplit, cb, ncols, Vk, ldv, noise, B ? B + (int64_t)k0 * ldb : nullptr,
            ldb, O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("tcd_reduce_kernel");
        k0 += ncols;
    }
}

}  // namespace kpcg
