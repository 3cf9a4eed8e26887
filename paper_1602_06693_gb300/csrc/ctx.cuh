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
    DevBuf<double> R64, Q64, Bblk, Sblk, G, colscale;
    DevBuf<float> W32;
    DevBuf<double> partial;
    DevBuf<double> scal;
    DevBuf<int> iscal;
    int* hflags = nullptr;  // pinned host [active, broken]
    std::string err;

    double c0_64() const { return std::log(s2); }
    float c0_32() const { return (float)(std::log(s2) * kLog2e); }
};

// Tensor-core K.V on the handle's inputs (kv_tc.cu).
void kv_tc_apply(Ctx& h, const float* V, int64_t ldv, int c, float* O, int64_t ldo);

}  // namespace kpcg
