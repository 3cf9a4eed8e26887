// Warm-start network: Linear(in,h1)-tanh-Linear(h1,h2)-tanh-Linear(h2,out),
// trained with Adam on mean squared error, run in FP32 (training) or with
// BF16 weights and inputs and FP32 accumulation (inference).  It maps the
// standardized log-hyperparameters of a trajectory to coefficients c on a fixed
// Nystrom basis Z, whose expansion K(X,Z|theta) c is the initial iterate x0 of
// Algorithm 1 (the paper's PCG takes x0 as input, Sec. 2.1).
//
// Sizes are small (batch <= a few hundred, layers <= 1024), so every kernel is
// a plain SIMT loop; one training step (forward, loss, backward, Adam) is
// captured once into a CUDA graph and replayed for the epochs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "kpcg_internal.cuh"

namespace kpcg {
namespace {

struct Layout {
    int in, h1, h2, out;
    size_t oW1, ob1, oW2, ob2, oW3, ob3, total;
    void build() {
        size_t o = 0;
        oW1 = o; o += (size_t)h1 * in;
        ob1 = o; o += h1;
        oW2 = o; o += (size_t)h2 * h1;
        ob2 = o; o += h2;
        oW3 = o; o += (size_t)out * h2;
        ob3 = o; o += out;
        total = o;
    }
};

// Y[b][o] = act(bias[o] + sum_i X[b][i] W[o][i]); one CTA per batch row.
template <typename TW>
__global__ void linear_fwd_kernel(const float* __restrict__ X, int I, const TW* __restrict__ W,
                                  const TW* __restrict__ bias, int O, float* __restrict__ Y,
                                  int act, int round_in_bf16) {
    extern __shared__ float xs[];
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        float v = X[(size_t)b * I + i];
        if (round_in_bf16) v = __bfloat162float(__float2bfloat16(v));
        xs[i] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        const TW* w = W + (size_t)o * I;
        float acc = (float)bias[o];
        for (int i = 0; i < I; ++i) acc = fmaf(xs[i], (float)w[i], acc);
        Y[(size_t)b * O + o] = act ? tanhf(acc) : acc;
    }
}
template <>
__global__ void linear_fwd_kernel<__nv_bfloat16>(const float* __restrict__ X, int I,
                                                 const __nv_bfloat16* __restrict__ W,
                                                 const __nv_bfloat16* __restrict__ bias, int O,
                                                 float* __restrict__ Y, int act,
                                                 int round_in_bf16) {
    extern __shared__ float xs[];
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        float v = X[(size_t)b * I + i];
        if (round_in_bf16) v = __bfloat162float(__float2bfloat16(v));
        xs[i] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        const __nv_bfloat16* w = W + (size_t)o * I;
        float acc = __bfloat162float(bias[o]);
        for (int i = 0; i < I; ++i) acc = fmaf(xs[i], __bfloat162float(w[i]), acc);
        Y[(size_t)b * O + o] = act ? tanhf(acc) : acc;
    }
}

// dY = 2 (Y - T) / (B O); loss = mean (Y - T)^2, one CTA, fixed-order reduction.
__global__ void mse_kernel(const float* __restrict__ Y, const float* __restrict__ T, int B, int O,
                           float* __restrict__ dY, float* __restrict__ loss) {
    __shared__ double sh[1024];
    const int N = B * O;
    const float scale = 2.0f / (float)N;
    double s = 0.0;
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        const float r = Y[e] - T[e];
        dY[e] = scale * r;
        s += (double)r * (double)r;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(sh[0] / (double)N);
}

// dX[b][i] = (sum_o dY[b][o] W[o][i]) * (1 - A[b][i]^2) (tanh derivative of
// the layer input A), one CTA per batch row.
__global__ void linear_bwd_data_kernel(const float* __restrict__ dY, int O,
                                       const float* __restrict__ W, int I,
                                       const float* __restrict__ A, float* __restrict__ dX) {
    extern __shared__ float dys[];
    const int b = blockIdx.x;
    for (int o = threadIdx.x; o < O; o += blockDim.x) dys[o] = dY[(size_t)b * O + o];
    __syncthreads();
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        float acc = 0.f;
        for (int o = 0; o < O; ++o) acc = fmaf(dys[o], W[(size_t)o * I + i], acc);
        const float a = A[(size_t)b * I + i];
        dX[(size_t)b * I + i] = acc * (1.f - a * a);
    }
}

// dW[o][i] = sum_b dY[b][o] X[b][i], db[o] = sum_b dY[b][o].
__global__ void linear_bwd_weight_kernel(const float* __restrict__ dY, int O,
                                         const float* __restrict__ X, int I, int B,
                                         float* __restrict__ dW, float* __restrict__ db) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = (int64_t)O * I;
    if (e < nw) {
        const int o = (int)(e / I), i = (int)(e % I);
        float acc = 0.f;
        for (int b = 0; b < B; ++b) acc = fmaf(dY[(size_t)b * O + o], X[(size_t)b * I + i], acc);
        dW[e] = acc;
    } else if (e < nw + O) {
        const int o = (int)(e - nw);
        float acc = 0.f;
        for (int b = 0; b < B; ++b) acc += dY[(size_t)b * O + o];
        db[o] = acc;
    }
}

// Adam with bias correction; state[0] = t, state[1] = beta1^t, state[2] = beta2^t
// advanced by one thread of the first CTA before the update of this step.
__global__ void adam_tick_kernel(float* state, float beta1, float beta2) {
    state[0] += 1.f;
    state[1] *= beta1;
    state[2] *= beta2;
}
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G,
                            float* __restrict__ M, float* __restrict__ V, size_t n,
                            const float* __restrict__ state, float lr, float beta1, float beta2,
                            float eps) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float g = G[e];
    const float m = beta1 * M[e] + (1.f - beta1) * g;
    const float v = beta2 * V[e] + (1.f - beta2) * g * g;
    M[e] = m;
    V[e] = v;
    const float mhat = m / (1.f - state[1]);
    const float vhat = v / (1.f - state[2]);
    P[e] -= lr * mhat / (sqrtf(vhat) + eps);
}

__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b,
                               size_t n) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = __float2bfloat16(a[e]);
}

unsigned blocks_for(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace kpcg

struct kpcg_mlp {
    kpcg::Layout L{};
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    kpcg::DevBuf<float> P, G, M, V, state, A1, A2, Y, dY, d2, d1, loss;
    kpcg::DevBuf<__nv_bfloat16> Pb;
    bool bf16_valid = false;
    // captured training step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const float* g_in = nullptr;
    const float* g_tg = nullptr;
    int g_batch = -1;
    float g_lr = 0.f;
    std::string err;
};

namespace kpcg {
static thread_local std::string g_mlp_err;

static void mlp_forward_fp32(kpcg_mlp& m, const float* X, int B, float* out) {
    const Layout& L = m.L;
    cudaStream_t st = m.stream;
    const float* P = m.P.p;
    linear_fwd_kernel<float><<<B, 256, sizeof(float) * L.in, st>>>(X, L.in, P + L.oW1, P + L.ob1,
                                                                  L.h1, m.A1.p, 1, 0);
    KPCG_LAUNCHED("linear_fwd_kernel");
    linear_fwd_kernel<float><<<B, 256, sizeof(float) * L.h1, st>>>(m.A1.p, L.h1, P + L.oW2,
                                                                  P + L.ob2, L.h2, m.A2.p, 1, 0);
    KPCG_LAUNCHED("linear_fwd_kernel");
    linear_fwd_kernel<float><<<B, 256, sizeof(float) * L.h2, st>>>(m.A2.p, L.h2, P + L.oW3,
                                                                  P + L.ob3, L.out, out, 0, 0);
    KPCG_LAUNCHED("linear_fwd_kernel");
}

// Forward, loss, backward into m.G; X (B x in), T (B x out).
static void mlp_grad_step(kpcg_mlp& m, const float* X, const float* T, int B) {
    const Layout& L = m.L;
    cudaStream_t st = m.stream;
    mlp_forward_fp32(m, X, B, m.Y.p);
    mse_kernel<<<1, 1024, 0, st>>>(m.Y.p, T, B, L.out, m.dY.p, m.loss.p);
    KPCG_LAUNCHED("mse_kernel");
    const float* P = m.P.p;
    float* G = m.G.p;
    // layer 3
    linear_bwd_weight_kernel<<<blocks_for((size_t)L.out * L.h2 + L.out), 256, 0, st>>>(
        m.dY.p, L.out, m.A2.p, L.h2, B, G + L.oW3, G + L.ob3);
    KPCG_LAUNCHED("linear_bwd_weight_kernel");
    linear_bwd_data_kernel<<<B, 256, sizeof(float) * L.out, st>>>(m.dY.p, L.out, P + L.oW3, L.h2,
                                                                 m.A2.p, m.d2.p);
    KPCG_LAUNCHED("linear_bwd_data_kernel");
    // layer 2
    linear_bwd_weight_kernel<<<blocks_for((size_t)L.h2 * L.h1 + L.h2), 256, 0, st>>>(
        m.d2.p, L.h2, m.A1.p, L.h1, B, G + L.oW2, G + L.ob2);
    KPCG_LAUNCHED("linear_bwd_weight_kernel");
    linear_bwd_data_kernel<<<B, 256, sizeof(float) * L.h2, st>>>(m.d2.p, L.h2, P + L.oW2, L.h1,
                                                                m.A1.p, m.d1.p);
    KPCG_LAUNCHED("linear_bwd_data_kernel");
    // layer 1
    linear_bwd_weight_kernel<<<blocks_for((size_t)L.h1 * L.in + L.h1), 256, 0, st>>>(
        m.d1.p, L.h1, X, L.in, B, G + L.oW1, G + L.ob1);
    KPCG_LAUNCHED("linear_bwd_weight_kernel");
}

static void mlp_adam(kpcg_mlp& m, float lr) {
    cudaStream_t st = m.stream;
    adam_tick_kernel<<<1, 1, 0, st>>>(m.state.p, 0.9f, 0.999f);
    KPCG_LAUNCHED("adam_tick_kernel");
    adam_kernel<<<blocks_for(m.L.total), 256, 0, st>>>(m.P.p, m.G.p, m.M.p, m.V.p, m.L.total,
                                                       m.state.p, lr, 0.9f, 0.999f, 1e-8f);
    KPCG_LAUNCHED("adam_kernel");
}
}  // namespace kpcg

using kpcg::fail;

#define MLP_GUARD(mp, ...)                         \
    try {                                          \
        __VA_ARGS__;                               \
    } catch (const kpcg::Error& e) {               \
        if (mp) (mp)->err = e.msg;                 \
        else kpcg::g_mlp_err = e.msg;              \
        return e.status;                           \
    }

extern "C" {

kpcg_status kpcg_mlp_create(int32_t n_in, int32_t h1, int32_t h2, int32_t n_out,
                            const float* params, int32_t max_batch, void* stream,
                            kpcg_mlp_t* out) {
    kpcg_mlp* m = nullptr;
    try {
        if (!out || !params) fail(KPCG_ERR_ARG, "NULL argument");
        *out = nullptr;
        if (n_in < 1 || h1 < 1 || h2 < 1 || n_out < 1 || n_in > 1024 || h1 > 1024 || h2 > 1024 ||
            n_out > 4096 || max_batch < 1 || max_batch > 4096)
            fail(KPCG_ERR_ARG, "layer sizes must be in [1, 1024] (output [1, 4096]), batch in [1, 4096]");
        m = new kpcg_mlp();
        m->L = kpcg::Layout{n_in, h1, h2, n_out};
        m->L.build();
        m->max_batch = max_batch;
        m->stream = (cudaStream_t)stream;
        const size_t T = m->L.total;
        m->P.need(T);
        m->G.need(T);
        m->M.need(T);
        m->V.need(T);
        m->state.need(3);
        m->A1.need((size_t)max_batch * h1);
        m->A2.need((size_t)max_batch * h2);
        m->Y.need((size_t)max_batch * n_out);
        m->dY.need((size_t)max_batch * n_out);
        m->d2.need((size_t)max_batch * h2);
        m->d1.need((size_t)max_batch * h1);
        m->loss.need(1);
        cudaStream_t st = m->stream;
        KPCG_CUDA(cudaMemcpyAsync(m->P.p, params, sizeof(float) * T, cudaMemcpyHostToDevice, st));
        KPCG_CUDA(cudaMemsetAsync(m->M.p, 0, sizeof(float) * T, st));
        KPCG_CUDA(cudaMemsetAsync(m->V.p, 0, sizeof(float) * T, st));
        const float s0[3] = {0.f, 1.f, 1.f};
        KPCG_CUDA(cudaMemcpyAsync(m->state.p, s0, sizeof(s0), cudaMemcpyHostToDevice, st));
        KPCG_CUDA(cudaStreamSynchronize(st));
        *out = m;
        return KPCG_OK;
    } catch (const kpcg::Error& e) {
        kpcg::g_mlp_err = e.msg;
        delete m;
        return e.status;
    }
}

kpcg_status kpcg_mlp_forward(kpcg_mlp_t m, const float* inputs, int32_t batch, float* out,
                             int32_t bf16) {
    if (!m) return KPCG_ERR_ARG;
    MLP_GUARD(m, {
        if (!inputs || !out) fail(KPCG_ERR_ARG, "NULL argument");
        if (batch < 1 || batch > m->max_batch) fail(KPCG_ERR_ARG, "batch out of range");
        cudaStream_t st = m->stream;
        if (!bf16) {
            kpcg::mlp_forward_fp32(*m, inputs, batch, out);
        } else {
            const kpcg::Layout& L = m->L;
            if (!m->bf16_valid) {
                m->Pb.need(L.total);
                kpcg::to_bf16_kernel<<<kpcg::blocks_for(L.total), 256, 0, st>>>(m->P.p, m->Pb.p,
                                                                               L.total);
                KPCG_LAUNCHED("to_bf16_kernel");
                m->bf16_valid = true;
            }
            const __nv_bfloat16* P = m->Pb.p;
            kpcg::linear_fwd_kernel<__nv_bfloat16><<<batch, 256, sizeof(float) * L.in, st>>>(
                inputs, L.in, P + L.oW1, P + L.ob1, L.h1, m->A1.p, 1, 1);
            KPCG_LAUNCHED("linear_fwd_kernel");
            kpcg::linear_fwd_kernel<__nv_bfloat16><<<batch, 256, sizeof(float) * L.h1, st>>>(
                m->A1.p, L.h1, P + L.oW2, P + L.ob2, L.h2, m->A2.p, 1, 1);
            KPCG_LAUNCHED("linear_fwd_kernel");
            kpcg::linear_fwd_kernel<__nv_bfloat16><<<batch, 256, sizeof(float) * L.h2, st>>>(
                m->A2.p, L.h2, P + L.oW3, P + L.ob3, L.out, out, 0, 1);
            KPCG_LAUNCHED("linear_fwd_kernel");
        }
        KPCG_CUDA(cudaStreamSynchronize(st));
    });
    return KPCG_OK;
}

kpcg_status kpcg_mlp_grad(kpcg_mlp_t m, const float* inputs, const float* targets, int32_t batch,
                          float* grads, float* loss_host) {
    if (!m) return KPCG_ERR_ARG;
    MLP_GUARD(m, {
        if (!inputs || !targets || !grads) fail(KPCG_ERR_ARG, "NULL argument");
        if (batch < 1 || batch > m->max_batch) fail(KPCG_ERR_ARG, "batch out of range");
        kpcg::mlp_grad_step(*m, inputs, targets, batch);
        KPCG_CUDA(cudaMemcpyAsync(grads, m->G.p, sizeof(float) * m->L.total,
                                  cudaMemcpyDeviceToDevice, m->stream));
        if (loss_host)
            KPCG_CUDA(cudaMemcpyAsync(loss_host, m->loss.p, sizeof(float), cudaMemcpyDeviceToHost,
                                      m->stream));
        KPCG_CUDA(cudaStreamSynchronize(m->stream));
    });
    return KPCG_OK;
}

kpcg_status kpcg_mlp_train(kpcg_mlp_t m, const float* inputs, const float* targets, int32_t batch,
                           int32_t epochs, float lr, float* loss_host) {
    if (!m) return KPCG_ERR_ARG;
    MLP_GUARD(m, {
        if (!inputs || !targets) fail(KPCG_ERR_ARG, "NULL argument");
        if (batch < 1 || batch > m->max_batch || epochs < 0) fail(KPCG_ERR_ARG, "bad sizes");
        if (!(lr > 0.f)) fail(KPCG_ERR_ARG, "lr must be > 0");
        cudaStream_t st = m->stream;
        // capture one full-batch step once per (inputs, targets, batch, lr)
        if (!m->exec || m->g_in != inputs || m->g_tg != targets || m->g_batch != batch ||
            m->g_lr != lr) {
            if (m->exec) cudaGraphExecDestroy(m->exec);
            if (m->graph) cudaGraphDestroy(m->graph);
            m->exec = nullptr;
            m->graph = nullptr;
            cudaStream_t cs;
            KPCG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaStream_t saved = m->stream;
            m->stream = cs;
            KPCG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            try {
                kpcg::mlp_grad_step(*m, inputs, targets, batch);
                kpcg::mlp_adam(*m, lr);
            } catch (...) {
                cudaGraph_t g;
                cudaStreamEndCapture(cs, &g);
                if (g) cudaGraphDestroy(g);
                m->stream = saved;
                cudaStreamDestroy(cs);
                throw;
            }
            KPCG_CUDA(cudaStreamEndCapture(cs, &m->graph));
            m->stream = saved;
            KPCG_CUDA(cudaStreamDestroy(cs));
            KPCG_CUDA(cudaGraphInstantiate(&m->exec, m->graph, 0));
            m->g_in = inputs;
            m->g_tg = targets;
            m->g_batch = batch;
            m->g_lr = lr;
        }
        for (int e = 0; e < epochs; ++e) KPCG_CUDA(cudaGraphLaunch(m->exec, st));
        m->bf16_valid = false;
        if (loss_host)
            KPCG_CUDA(cudaMemcpyAsync(loss_host, m->loss.p, sizeof(float), cudaMemcpyDeviceToHost,
                                      st));
        KPCG_CUDA(cudaStreamSynchronize(st));
    });
    return KPCG_OK;
}

kpcg_status kpcg_mlp_get_params(kpcg_mlp_t m, float* params_host) {
    if (!m) return KPCG_ERR_ARG;
    MLP_GUARD(m, {
        if (!params_host) fail(KPCG_ERR_ARG, "NULL argument");
        KPCG_CUDA(cudaMemcpyAsync(params_host, m->P.p, sizeof(float) * m->L.total,
                                  cudaMemcpyDeviceToHost, m->stream));
        KPCG_CUDA(cudaStreamSynchronize(m->stream));
    });
    return KPCG_OK;
}

void kpcg_mlp_destroy(kpcg_mlp_t m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->graph) cudaGraphDestroy(m->graph);
    delete m;
}

const char* kpcg_mlp_last_error(kpcg_mlp_t m) {
    if (!m) return kpcg::g_mlp_err.c_str();
    return m->err.c_str();
}

}  // extern "C"
