// Double-float arithmetic on the FP32 pipe (unevaluated sums hi + lo of two
// FP32 numbers, ~44 bits): Knuth's TwoSum accumulation and the table-driven
// exp2 of P. T. P. Tang ("Table-driven implementation of the exponential
// function", 1989) with a 257-entry double-float table of 2^(j/256) (and a
// 1024-entry one of 2^(j/1024)) built on the host in FP64.  Shared by the
// double-float kernels (kv_df.cu, kv_tcd.cu).
#pragma once

#include <cuda_runtime.h>

namespace kpcg {
namespace {

constexpr int NTAB = 257;  // 2^(j/256), j = -128..128
constexpr float kLn2Hi = 0.6931471824645996f;     // fl(ln 2)
constexpr float kLn2Lo = -1.9046542121259336e-09f;  // fl(ln 2 - kLn2Hi)

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

// Fold the compensation into the sum (Fast2Sum), keeping C small so its own
// FP32 roundings stay below 2^-48 of the sum over long accumulations.
__device__ __forceinline__ void df_renorm(float& S, float& C) {
    const float s = S + C;
    C = C - (s - S);
    S = s;
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

constexpr int NTAB1K = 1024;  // 2^(j/1024), j = 0..1023

// 2^(ah + al) as a double-float, the same method with a finer table (for
// the symmetric tensor-core kernel).  (ah, al) need not be normalised.
// Arguments below -125 are clamped there
// (the result is then 2^-125 instead of zero: far below any entry that
// matters against s^2).  a = m/1024 + r with m = rint(1024 a), read off the
// mantissa of 1024 a + 1.5 * 2^23 (no float-to-int conversion), |r| <=
// 2^-11 exactly; 2^a = 2^(m >> 10) * 2^((m & 1023)/1024) * e^t with t = (r +
// al) ln 2 as th + tl and e^t = 1 + t + t^2 (1/2 + t/6) (the next term is
// below 2^-52; th^2 rounds at 2^-47).
__device__ __forceinline__ DF df_exp2_1k(float ah, float al, const float2* __restrict__ tab) {
    // renormalise: the low part of a sum of level accumulators can exceed
    // half an ulp of the high part, and t below must stay within 2^-11
    const float s = ah + al;
    al = al - (s - ah);
    ah = fmaxf(s, -125.f);
    const float t = fmaf(ah, 1024.f, 12582912.f);     // 1.5 * 2^23 + m
    const int mi = __float_as_int(t) - 0x4B400000;    // m
    const float mf = t - 12582912.f;                   // m, exact
    const float rh = fmaf(mf, -0.0009765625f, ah);     // exact, |rh| <= 2^-11
    const float th = rh * kLn2Hi;
    float tl = fmaf(rh, kLn2Hi, -th);
    tl = fmaf(rh, kLn2Lo, tl);
    tl = fmaf(al, kLn2Hi, tl);
    const float w = fmaf(th, 0.16666666666666666f, 0.5f);
    float q = fmaf(th * th, w, tl);
    q = fmaf(th, tl, q);
    const float uh = 1.f + th;
    const float ul = ((1.f - uh) + th) + q;
    const float2 T = tab[mi & (NTAB1K - 1)];
    const float sc = __int_as_float(((mi >> 10) + 127) << 23);
    const float ph = T.x * uh;
    float pl = fmaf(T.x, uh, -ph);
    pl = fmaf(T.x, ul, pl);
    pl = fmaf(T.y, uh, pl);
    DF r;
    r.h = ph * sc;
    r.l = pl * sc;
    return r;
}

}  // namespace
}  // namespace kpcg
