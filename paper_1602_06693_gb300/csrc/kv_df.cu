// Double-float K.V: FP64-class kernel products on the FP32 pipe.
//
// GB300 issues FP32 at 64 times its FP64 rate, and an FP64 K.V at n = 65536
// is bound by that FP64 rate.  This kernel carries every quantity of an entry
// K_ij = s^2 exp(-1/2 sum_r (x_ir - x_jr)^2 / l_r^2) (Eq. 1) as an unevaluated
// sum of two FP32 numbers (hi + lo), which keeps about 44 bits:
//
//  * Inputs.  x' = (x - mu) / l * sqrt(log2(e)/2) (FP64) is split per
//    dimension r into hi, a multiple of 2^(k_r - 23) with |x'| < 2^k_r (so
//    hi_i - hi_j is exact in FP32), lo = fl(x' - hi) and lo2 = fl(x' - hi - lo):
//    the three parts hold the FP64 value exactly, so the only per-point error
//    is the FP64 rounding of x' itself.  (With two parts, the 2^-48 rounding of
//    lo is a per-point, hence structured, perturbation of K; multiplied by a
//    solution with |alpha| >> |y| it limited the residual to about 1e-7.)
//  * Squared distance.  delta = D + E with D = hi_i - hi_j exact, E = (lo_i -
//    lo_j) + (lo2_i - lo2_j); delta^2 = D*D (split exactly by an FMA,
//    "TwoProduct") + 2 D E + E^2,
//    accumulated into the exponent a = log2(s^2) - |x'_i - x'_j|^2 with Knuth's
//    TwoSum, so no rounding of the running sum is lost.
//  * exp2 of a double-float (table-driven method of P. T. P. Tang, "Table-
//    driven implementation of the exponential function", 1989): a = k + j/256
//    + r, 2^a = 2^k * 2^(j/256) * e^(r ln 2); the 257 values 2^(j/256) are a
//    double-float table computed on the host in FP64, e^t for |t| < 0.0014 is
//    1 + t + t^2 (1/2 + t (1/6 + t/24)) with the linear part in double-float.
//  * Contraction.  V (FP64) enters as hi + lo; products are split exactly and
//    summed with TwoSum (Ogita-Rump-Oishi style), partial sums leave as FP64.
//
// Rows: one per thread; column tiles of the operands staged in shared memory;
// column ranges split across CTAs and added in FP64 by a second kernel in a
// fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"

namespace kpcg {
namespace {

constexpr int KT = 256;
constexpr int TJ = 64;
constexpr int NTAB = 257;  // 2^(j/256), j = -128..128
constexpr float kLn2Hi = 0.6931471824645996f;     // fl(ln 2)
constexpr float kLn2Lo = -1.9046542121259336e-09f;  // fl(ln 2 - kLn2Hi)

int sm_count_df() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        if (cached <= 0) cached = 148;
    }
    return cached;
}

struct DF {
    float h, l;
};

// a := a - (P + Pe) with TwoSum on the high parts.
__device__ __forceinline__ void df_sub(float& ah, float& al, float P, float Pe) {
    const float s = ah - P;
    const float bb = s - ah;
    const float err = (ah - (s - bb)) + (-P - bb);
    ah = s;
    al += err - Pe;
}
// (S, C) += (P, Pe) with TwoSum on the high parts.
__device__ __forceinline__ void df_acc(float& S, float& C, float P, float Pe) {
    const float s = S + P;
    const float bb = s - S;
    const float err = (S - (s - bb)) + (P - bb);
    S = s;
    C += err + Pe;
}

// 2^(ah + al) as a double-float; zero below 2^-126.
__device__ __forceinline__ DF df_exp2(float ah, float al, const float2* __restrict__ tab) {
    // renormalise
    const float s = ah + al;
    al = al - (s - ah);
    ah = s;
    const float k = rintf(ah);
    const float fh = ah - k;               // exact, |fh| <= 1/2
    const float jf = rintf(fh * 256.f);
    const float rh = fmaf(jf, -0.00390625f, fh);  // exact, |rh| <= 1/512
    // t = (rh + al) ln 2 as th + tl (TwoProduct on rh * ln2_hi)
    const float th = rh * kLn2Hi;
    float tl = fmaf(rh, kLn2Hi, -th);
    tl = fmaf(rh, kLn2Lo, tl);
    tl = fmaf(al, kLn2Hi, tl);
    // e^t - 1 - t = t^2 (1/2 + t (1/6 + t / 24)), t^2 split exactly
    const float w = fmaf(th, fmaf(th, 0.041666666666666664f, 0.16666666666666666f), 0.5f);
    const float p2 = th * th;
    const float p2e = fmaf(th, th, -p2);
    const float q = fmaf(p2, w, 0.5f * p2e);
    tl = fmaf(th, tl, tl + q);
    const float uh = 1.f + th;
    const float ul = ((1.f - uh) + th) + tl;
    const float2 T = tab[(int)jf + 128];
    const float ph = T.x * uh;
    float pl = fmaf(T.x, uh, -ph);
    pl = fmaf(T.x, ul, pl);
    pl = fmaf(T.y, uh, pl);
    DF r;
    if (k < -125.f) {
        r.h = 0.f;
        r.l = 0.f;
    } else {
        const float sc = __int_as_float(((int)k + 127) << 23);
        r.h = ph * sc;
        r.l = pl * sc;
    }
    return r;
}

template <int DP, int CB>
__global__ void __launch_bounds__(KT)
    kv_df_kernel(const float4* __restrict__ xs, int64_t n, float c0h, float c0l,
                 const double* __restrict__ V, int64_t ldv, int ncols,
                 const float2* __restrict__ gtab, double* __restrict__ part, int64_t ldp,
                 int64_t cps) {
    __shared__ float2 tab[NTAB];
    __shared__ float4 sx[TJ * DP];
    __shared__ float2 sv[TJ * CB];
    for (int e = threadIdx.x; e < NTAB; e += KT) tab[e] = gtab[e];
    const int64_t i = (int64_t)blockIdx.x * KT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * cps;
    const int64_t j1 = min(n, j0 + cps);
    float4 xi[DP];
#pragma unroll
    for (int q = 0; q < DP; ++q) xi[q] = (i < n) ? xs[i * DP + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    float S[CB], C[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) S[k] = C[k] = 0.f;
    for (int64_t jt = j0; jt < j1; jt += TJ) {
        const int jn = (int)min((int64_t)TJ, j1 - jt);
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * DP; e += KT) {
            const int jj = e / DP;
            sx[e] = (jj < jn) ? xs[(jt + jj) * DP + (e - jj * DP)] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = threadIdx.x; e < TJ * CB; e += KT) {
            const int k = e / TJ, jj = e - k * TJ;
            double v = (jj < jn && k < ncols) ? V[(jt + jj) + (int64_t)k * ldv] : 0.0;
            const float vh = (float)v;
            sv[jj * CB + k] = make_float2(vh, (float)(v - (double)vh));
        }
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            float ah = c0h, al = c0l;
#pragma unroll
            for (int q = 0; q < DP; ++q) {
                const float4 xj = sx[jj * DP + q];
                const float D = xi[q].x - xj.x;  // exact
                const float E = (xi[q].y - xj.y) + (xi[q].z - xj.z);
                const float P = D * D;
                float Pe = fmaf(D, D, -P);
                Pe = fmaf(2.f * D, E, Pe);
                Pe = fmaf(E, E, Pe);
                df_sub(ah, al, P, Pe);
            }
            const DF e = df_exp2(ah, al, tab);
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const float2 v = sv[jj * CB + k];
                const float P = e.h * v.x;
                float Pe = fmaf(e.h, v.x, -P);
                Pe = fmaf(e.h, v.y, Pe);
                Pe = fmaf(e.l, v.x, Pe);
                df_acc(S[k], C[k], P, Pe);
            }
        }
    }
    if (i < n) {
#pragma unroll
        for (int k = 0; k < CB; ++k)
            if (k < ncols) part[((int64_t)blockIdx.y * CB + k) * ldp + i] = (double)S[k] + (double)C[k];
    }
}

__global__ void kv_df_reduce_kernel(const double* __restrict__ part, int64_t ldp, int nsplit,
                                    int cb, int ncols, const double* __restrict__ V, int64_t ldv,
                                    double noise, const double* __restrict__ B, int64_t ldb,
                                    double* __restrict__ O, int64_t ldo, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= n || k >= ncols) return;
    double s = noise * V[i + (int64_t)k * ldv];
    for (int sp = 0; sp < nsplit; ++sp) s += part[((int64_t)sp * cb + k) * ldp + i];
    O[i + (int64_t)k * ldo] = B ? (B[i + (int64_t)k * ldb] - s) : s;
}

// Column-wise max |x'| (FP64) to pick the grid of the hi parts.
__global__ void colmax_kernel(const double* __restrict__ xs64, int64_t n, int dp,
                              double* __restrict__ out) {
    __shared__ double sh[256];
    const int q = blockIdx.x;
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(xs64[i * dp + q]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

// hi = x' rounded to the grid 2^(k_r - 23), lo = fl(x' - hi), lo2 = x' - hi - lo.
__global__ void df_prep_kernel(const double* __restrict__ xs64, int64_t n, int dp, double scale,
                               const double* __restrict__ grid, float4* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * dp) return;
    const int q = (int)(e % dp);
    const double x = xs64[e] * scale;
    const double g = grid[q];
    const double hi = rint(x / g) * g;
    const float lo = (float)(x - hi);
    const float lo2 = (float)(x - hi - (double)lo);
    out[e] = make_float4((float)hi, lo, lo2, 0.f);
}

struct DfSplit {
    int nrb, nsplit;
    int64_t cps, ldp;
};

DfSplit df_plan(int64_t n) {
    DfSplit s;
    s.nrb = (int)((n + KT - 1) / KT);
    const int64_t target = (int64_t)sm_count_df() * 8;
    int64_t ns = (target + s.nrb - 1) / s.nrb;
    ns = std::max<int64_t>(1, std::min(ns, (n + TJ - 1) / TJ));
    int64_t cps = (n + ns - 1) / ns;
    cps = ((cps + TJ - 1) / TJ) * TJ;
    s.cps = cps;
    s.nsplit = (int)((n + cps - 1) / cps);
    s.ldp = ((n + 31) / 32) * 32;
    return s;
}

template <int DP, int CB>
void df_launch(const float4* xs, int64_t n, float c0h, float c0l, const double* V, int64_t ldv,
               int ncols, const float2* tab, double* part, const DfSplit& s, cudaStream_t st) {
    kv_df_kernel<DP, CB><<<dim3(s.nrb, s.nsplit), KT, 0, st>>>(xs, n, c0h, c0l, V, ldv, ncols,
                                                               tab, part, s.ldp, s.cps);
    KPCG_LAUNCHED("kv_df_kernel");
}

template <int DP>
void df_launch_cb(int cb, const float4* xs, int64_t n, float c0h, float c0l, const double* V,
                  int64_t ldv, int ncols, const float2* tab, double* part, const DfSplit& s,
                  cudaStream_t st) {
    switch (cb) {
        case 1: df_launch<DP, 1>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st); break;
        case 2: df_launch<DP, 2>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st); break;
        case 4: df_launch<DP, 4>(xs, n, c0h, c0l, V, ldv, ncols, tab, part, s, st); break;
        default: fail(KPCG_ERR_ARG, "internal: bad column block");
    }
}

}  // namespace

// Refresh the double-float inputs of the handle after theta changed.
static void df_prepare(Ctx& h) {
    if (h.df_version == h.theta_version) return;
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    if (!h.df_tab.p) {
        std::vector<float2> t(NTAB);
        for (int j = -128; j <= 128; ++j) {
            const double v = std::exp2((double)j / 256.0);
            const float hi = (float)v;
            t[j + 128] = make_float2(hi, (float)(v - (double)hi));
        }
        h.df_tab.need(NTAB);
        KPCG_CUDA(cudaMemcpyAsync(h.df_tab.p, t.data(), sizeof(float2) * NTAB,
                                  cudaMemcpyHostToDevice, st));
    }
    // x' in the exp2 scaling: xs64 * sqrt(log2 e)
    const double scale = std::sqrt(kLog2e);
    double* mx = h.df_grid.need((size_t)2 * h.dp);
    colmax_kernel<<<h.dp, 256, 0, st>>>(h.xs64.p, n, h.dp, mx);
    KPCG_LAUNCHED("colmax_kernel");
    std::vector<double> hm((size_t)h.dp), grid((size_t)h.dp);
    KPCG_CUDA(cudaMemcpyAsync(hm.data(), mx, sizeof(double) * h.dp, cudaMemcpyDeviceToHost, st));
    KPCG_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < h.dp; ++q) {
        const double m = hm[q] * scale;
        int k = 0;
        if (m > 0.0) k = (int)std::floor(std::log2(m)) + 1;  // |x'| < 2^k
        grid[q] = std::ldexp(1.0, k - 23);
    }
    KPCG_CUDA(cudaMemcpyAsync(mx + h.dp, grid.data(), sizeof(double) * h.dp,
                              cudaMemcpyHostToDevice, st));
    float4* xdf = reinterpret_cast<float4*>(h.xdf.need((size_t)n * h.dp * 4));
    df_prep_kernel<<<(unsigned)((n * h.dp + 255) / 256), 256, 0, st>>>(h.xs64.p, n, h.dp, scale,
                                                                       mx + h.dp, xdf);
    KPCG_LAUNCHED("df_prep_kernel");
    const double c0 = std::log2(h.s2);
    h.df_c0h = (float)c0;
    h.df_c0l = (float)(c0 - (double)h.df_c0h);
    h.df_version = h.theta_version;
}

void kv_df(Ctx& h, const double* V, int64_t ldv, int c, const double* B, int64_t ldb, double* O,
           int64_t ldo, double noise) {
    if (h.n <= 0 || c <= 0) return;
    df_prepare(h);
    cudaStream_t st = h.stream;
    const int64_t n = h.n;
    const DfSplit s = df_plan(n);
    const int max_cb = 4;
    double* part = h.kvws.part64.need((size_t)s.nsplit * max_cb * s.ldp);
    const float4* xs = reinterpret_cast<const float4*>(h.xdf.p);
    const float2* tab = reinterpret_cast<const float2*>(h.df_tab.p);
    for (int k0 = 0; k0 < c;) {
        const int rem = c - k0;
        const int cb = rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        const int ncols = std::min(cb, rem);
        const double* Vk = V + (int64_t)k0 * ldv;
        switch (h.dp) {
            case 4: df_launch_cb<4>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 8: df_launch_cb<8>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 12: df_launch_cb<12>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 16: df_launch_cb<16>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            case 32: df_launch_cb<32>(cb, xs, n, h.df_c0h, h.df_c0l, Vk, ldv, ncols, tab, part, s, st); break;
            default: fail(KPCG_ERR_ARG, "unsupported padded dimension");
        }
        kv_df_reduce_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)ncols), 256, 0, st>>>(
            part, s.ldp, s.nsplit, cb, ncols, Vk, ldv, noise, B ? B + (int64_t)k0 * ldb : nullptr,
            ldb, O + (int64_t)k0 * ldo, ldo, n);
        KPCG_LAUNCHED("kv_df_reduce_kernel");
        k0 += ncols;
    }
}

}  // namespace kpcg
