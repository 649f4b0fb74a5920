// Surrogate network kernels: a multilayer perceptron 5 -> 128 -> 128 -> 128
// -> 128 -> 2 with SiLU on the hidden layers, BF16 weights and FP32
// accumulation, trained with Adam on FP32 master weights (the learned part
// that picks capillary numbers near breakup).
//
// Forward, backward, loss and optimiser are hand-written kernels.  The
// contractions are small (n x 128 x 128 per layer with n up to a few
// thousand samples, ~1e7 multiply-adds per step): a tiled FMA kernel with the
// weight tile and the input tile in shared memory finishes each in a few
// microseconds, so the tensor cores would not change the step time.
// Reductions over samples (weight gradients, loss) are deterministic: each
// block owns its output tile and loops over all samples in a fixed order.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"

namespace surr {

constexpr int NLAYER = 5;
constexpr int WIDTH[NLAYER + 1] = {5, 128, 128, 128, 128, 2};
constexpr int MAXW = 128;

// Parameter offsets in the flat FP32 vector: layer l holds W [fout][fin]
// then b [fout].
struct Offsets {
    int w[NLAYER], b[NLAYER], total;
    constexpr Offsets() : w(), b(), total(0) {
        int o = 0;
        for (int l = 0; l < NLAYER; ++l) {
            w[l] = o;
            o += WIDTH[l + 1] * WIDTH[l];
            b[l] = o;
            o += WIDTH[l + 1];
        }
        total = o;
    }
};
constexpr Offsets OFF{};

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// out_pre[n][fout] = in[n][fin] W^T + b; out_act = SiLU(out_pre) (hidden) or
// out_pre (last layer).  Block: 32 samples x 32 outputs, 256 threads, each
// thread 4 outputs of one sample.
constexpr int FT_S = 32, FT_O = 32;

__global__ void __launch_bounds__(256) k_linear_fwd(const float* __restrict__ in, int fin,
                                                    const __nv_bfloat16* __restrict__ W,
                                                    const float* __restrict__ b, int fout, int n,
                                                    float* __restrict__ pre,
                                                    float* __restrict__ act, int hidden) {
    __shared__ float sx[FT_S][MAXW + 1];
    __shared__ float sw[FT_O][MAXW + 1];
    const int s0 = blockIdx.x * FT_S, o0 = blockIdx.y * FT_O;
    for (int k = threadIdx.x; k < FT_S * fin; k += blockDim.x) {
        const int s = k / fin, i = k % fin;
        sx[s][i] = (s0 + s < n) ? in[(int64_t)(s0 + s) * fin + i] : 0.0f;
    }
    for (int k = threadIdx.x; k < FT_O * fin; k += blockDim.x) {
        const int o = k / fin, i = k % fin;
        sw[o][i] = (o0 + o < fout) ? __bfloat162float(W[(int64_t)(o0 + o) * fin + i]) : 0.0f;
    }
    __syncthreads();
    const int s = threadIdx.x / 8, og = threadIdx.x % 8;  // outputs og, og+8, og+16, og+24
    float acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = 0.0f;
    for (int i = 0; i < fin; ++i) {
        const float x = sx[s][i];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fmaf(x, sw[og + 8 * j][i], acc[j]);
    }
    if (s0 + s >= n) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int o = o0 + og + 8 * j;
        if (o >= fout) continue;
        const float z = acc[j] + b[o];
        pre[(int64_t)(s0 + s) * fout + o] = z;
        act[(int64_t)(s0 + s) * fout + o] = hidden ? silu(z) : z;
    }
}

// Gradient of the loss  mean((D - yD)^2) + mean(BCE(z, yB))  with respect to
// the two outputs, and the loss itself (one block, fixed-order reduction).
__global__ void k_loss_grad(const float* __restrict__ out, const float* __restrict__ yD,
                            const float* __restrict__ yB, int n, float* __restrict__ gout,
                            double* __restrict__ loss) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const float d = out[2 * s] - yD[s];
        const float z = out[2 * s + 1];
        const float y = yB[s];
        gout[2 * s] = 2.0f * d / n;
        gout[2 * s + 1] = (1.0f / (1.0f + expf(-z)) - y) / n;
        const double bce = fmax((double)z, 0.0) - (double)z * y + log1p(exp(-fabs((double)z)));
        acc += (double)d * d + bce;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / n;
}

// gin[n][fin] = (gpre[n][fout] W) * SiLU'(pre_in[n][fin])  (pre_in NULL: no
// activation factor).  Block: 32 samples x 32 inputs.
__global__ void __launch_bounds__(256) k_linear_bwd_in(const float* __restrict__ gpre, int fout,
                                                       const __nv_bfloat16* __restrict__ W,
                                                       int fin, int n,
                                                       const float* __restrict__ pre_in,
                                                       float* __restrict__ gin) {
    __shared__ float sg[FT_S][MAXW + 1];
    __shared__ float sw[MAXW][FT_O + 1];
    const int s0 = blockIdx.x * FT_S, i0 = blockIdx.y * FT_O;
    for (int k = threadIdx.x; k < FT_S * fout; k += blockDim.x) {
        const int s = k / fout, o = k % fout;
        sg[s][o] = (s0 + s < n) ? gpre[(int64_t)(s0 + s) * fout + o] : 0.0f;
    }
    for (int k = threadIdx.x; k < fout * FT_O; k += blockDim.x) {
        const int o = k / FT_O, i = k % FT_O;
        sw[o][i] = (i0 + i < fin) ? __bfloat162float(W[(int64_t)o * fin + i0 + i]) : 0.0f;
    }
    __syncthreads();
    const int s = threadIdx.x / 8, ig = threadIdx.x % 8;
    float acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = 0.0f;
    for (int o = 0; o < fout; ++o) {
        const float g = sg[s][o];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fmaf(g, sw[o][ig + 8 * j], acc[j]);
    }
    if (s0 + s >= n) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = i0 + ig + 8 * j;
        if (i >= fin) continue;
        float v = acc[j];
        if (pre_in) v *= silu_grad(pre_in[(int64_t)(s0 + s) * fin + i]);
        gin[(int64_t)(s0 + s) * fin + i] = v;
    }
}

// gW[fout][fin] = sum_s gpre[s][o] in[s][i]; gb[o] = sum_s gpre[s][o].
// Block: 32 outputs x 32 inputs (plus the bias column), loops over all
// samples in chunks of 64 (fixed order: deterministic).
constexpr int GT = 32, GCH = 64;

__global__ void __launch_bounds__(256) k_linear_bwd_w(const float* __restrict__ gpre, int fout,
                                                      const float* __restrict__ in, int fin,
                                                      int n, float* __restrict__ gW,
                                                      float* __restrict__ gb) {
    __shared__ float sg[GCH][GT + 1];
    __shared__ float sx[GCH][GT + 1];
    const int o0 = blockIdx.x * GT, i0 = blockIdx.y * GT;
    const int oi = threadIdx.x / 8;         // output row in the tile (0..31)
    const int ig = threadIdx.x % 8;         // inputs ig, ig+8, ig+16, ig+24
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float accb = 0.0f;
    for (int c0 = 0; c0 < n; c0 += GCH) {
        for (int k = threadIdx.x; k < GCH * GT; k += blockDim.x) {
            const int s = k / GT, j = k % GT;
            const bool ok = c0 + s < n;
            sg[s][j] = (ok && o0 + j < fout) ? gpre[(int64_t)(c0 + s) * fout + o0 + j] : 0.0f;
            sx[s][j] = (ok && i0 + j < fin) ? in[(int64_t)(c0 + s) * fin + i0 + j] : 0.0f;
        }
        __syncthreads();
        for (int s = 0; s < GCH; ++s) {
            const float g = sg[s][oi];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fmaf(g, sx[s][ig + 8 * j], acc[j]);
            accb += g;
        }
        __syncthreads();
    }
    const int o = o0 + oi;
    if (o >= fout) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = i0 + ig + 8 * j;
        if (i < fin) gW[(int64_t)o * fin + i] = acc[j];
    }
    if (blockIdx.y == 0 && ig == 0) gb[o] = accb;
}

// Adam with bias correction on the FP32 master parameters, then their BF16
// copies (weights only are used in BF16; biases stay FP32).  The step number
// is *t + 1, read on the device (k_to_bf16 advances *t after the step), so
// that one captured step can be replayed.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int count, float lr, float b1, float b2, float eps,
                       const long long* __restrict__ t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const double step = (double)(*t + 1);
    const float c1 = (float)(1.0 - pow((double)b1, step));
    const float c2 = (float)(1.0 - pow((double)b2, step));
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float mh = mk / c1, vh = vk / c2;
    p[k] -= lr * mh / (sqrtf(vh) + eps);
}

// BF16 copies of the parameters; `tick` (nullable): the Adam step counter,
// advanced by one.
__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int count,
                          long long* __restrict__ tick) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) q[k] = __float2bfloat16_rn(p[k]);
    if (tick && k == 0) *tick += 1;
}

}  // namespace surr

using namespace surr;

struct surr_ctx {
    float* params = nullptr;          // FP32 master parameters (flat)
    __nv_bfloat16* wq = nullptr;      // BF16 copies (flat, same offsets)
    float* grads = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    long long* adam_t = nullptr;      // Adam steps taken (device counter)
    // one captured training step (forward, backward, Adam, BF16 copies),
    // valid for n samples and learning rate lr with the current buffers
    cudaGraphExec_t step_graph = nullptr;
    int graph_n = 0;
    float graph_lr = 0.0f;
    cudaStream_t cap_stream = nullptr;
    int cap = 0;                      // samples the activation buffers hold
    float* x = nullptr;               // inputs [cap][5]
    float* pre[NLAYER] = {};          // pre-activations per layer [cap][fout]
    float* act[NLAYER] = {};          // activations per layer [cap][fout]
    float* gbuf[2] = {nullptr, nullptr};  // gradient ping-pong [cap][128]
    float* yD = nullptr;
    float* yB = nullptr;
    double* loss = nullptr;
    cudaStream_t stream = nullptr;
};

namespace {

int fail(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    cudaGetLastError();
    return LBM_ERR_CUDA;
}

void drop_step_graph(surr_ctx* c) {
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    c->step_graph = nullptr;
}

void free_batch(surr_ctx* c) {
    drop_step_graph(c);  // it refers to the activation buffers
    cudaFree(c->x);
    for (int l = 0; l < NLAYER; ++l) {
        cudaFree(c->pre[l]);
        cudaFree(c->act[l]);
        c->pre[l] = c->act[l] = nullptr;
    }
    cudaFree(c->gbuf[0]);
    cudaFree(c->gbuf[1]);
    cudaFree(c->yD);
    cudaFree(c->yB);
    c->x = c->gbuf[0] = c->gbuf[1] = c->yD = c->yB = nullptr;
    c->cap = 0;
}

int ensure_batch(surr_ctx* c, int n) {
    if (n <= c->cap) return LBM_OK;
    free_batch(c);
    bool ok = cudaMalloc(&c->x, sizeof(float) * n * WIDTH[0]) == cudaSuccess &&
              cudaMalloc(&c->gbuf[0], sizeof(float) * n * MAXW) == cudaSuccess &&
              cudaMalloc(&c->gbuf[1], sizeof(float) * n * MAXW) == cudaSuccess &&
              cudaMalloc(&c->yD, sizeof(float) * n) == cudaSuccess &&
              cudaMalloc(&c->yB, sizeof(float) * n) == cudaSuccess;
    for (int l = 0; l < NLAYER && ok; ++l)
        ok = cudaMalloc(&c->pre[l], sizeof(float) * n * WIDTH[l + 1]) == cudaSuccess &&
             cudaMalloc(&c->act[l], sizeof(float) * n * WIDTH[l + 1]) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(c);
        return LBM_ERR_NOMEM;
    }
    c->cap = n;
    return LBM_OK;
}

void refresh_bf16(surr_ctx* c, bool tick = false) {
    k_to_bf16<<<(OFF.total + 255) / 256, 256, 0, c->stream>>>(c->params, c->wq, OFF.total,
                                                              tick ? c->adam_t : nullptr);
}

void forward(surr_ctx* c, int n) {
    const float* in = c->x;
    for (int l = 0; l < NLAYER; ++l) {
        const int fin = WIDTH[l], fout = WIDTH[l + 1];
        dim3 grid((n + FT_S - 1) / FT_S, (fout + FT_O - 1) / FT_O);
        k_linear_fwd<<<grid, 256, 0, c->stream>>>(in, fin, c->wq + OFF.w[l], c->params + OFF.b[l],
                                                  fout, n, c->pre[l], c->act[l], l < NLAYER - 1);
        in = c->act[l];
    }
}

// Gradients of the loss for the n samples in the activation buffers into
// c->grads (needs forward first and yD, yB on the device).
void backward(surr_ctx* c, int n) {
    k_loss_grad<<<1, 256, 0, c->stream>>>(c->act[NLAYER - 1], c->yD, c->yB, n, c->gbuf[0], c->loss);
    int cur = 0;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const int fin = WIDTH[l], fout = WIDTH[l + 1];
        const float* in = l == 0 ? c->x : c->act[l - 1];
        dim3 gw((fout + GT - 1) / GT, (fin + GT - 1) / GT);
        k_linear_bwd_w<<<gw, 256, 0, c->stream>>>(c->gbuf[cur], fout, in, fin, n,
                                                  c->grads + OFF.w[l], c->grads + OFF.b[l]);
        if (l > 0) {
            dim3 gi((n + FT_S - 1) / FT_S, (fin + FT_O - 1) / FT_O);
            k_linear_bwd_in<<<gi, 256, 0, c->stream>>>(c->gbuf[cur], fout, c->wq + OFF.w[l], fin,
                                                        n, c->pre[l - 1], c->gbuf[1 - cur]);
            cur = 1 - cur;
        }
    }
}

// One Adam step on the n samples in the buffers.
void train_step(surr_ctx* c, int n, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    forward(c, n);
    backward(c, n);
    k_adam<<<(OFF.total + 255) / 256, 256, 0, c->stream>>>(c->params, c->grads, c->m, c->v,
                                                           OFF.total, lr, b1, b2, eps, c->adam_t);
    refresh_bf16(c, true);
}

// The step as a graph (captured on the private stream; replayed on c->stream).
int build_step_graph(surr_ctx* c, int n, float lr) {
    drop_step_graph(c);
    if (!c->cap_stream &&
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(cudaGetLastError());
    const cudaStream_t saved = c->stream;
    c->stream = c->cap_stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        train_step(c, n, lr);
        e = cudaStreamEndCapture(c->cap_stream, &g);
    }
    c->stream = saved;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->step_graph = nullptr;
        return fail(e);
    }
    c->graph_n = n;
    c->graph_lr = lr;
    return LBM_OK;
}

int upload_batch(surr_ctx* c, const float* X, const float* yD, const float* yB, int n) {
    int rc = ensure_batch(c, n);
    if (rc != LBM_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(c->x, X, sizeof(float) * n * WIDTH[0], cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess && yD)
        e = cudaMemcpyAsync(c->yD, yD, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && yB)
        e = cudaMemcpyAsync(c->yB, yB, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream);
    return fail(e);
}

// The body of surr_train (arguments checked).
int train_epochs(surr_ctx* c, const float* X, const float* yD, const float* yB, int n, int epochs,
                 float lr, double* loss_out) {
    int rc = upload_batch(c, X, yD, yB, n);
    if (rc != LBM_OK) return rc;
    // the step's launches are captured once and the graph replayed per epoch
    if (epochs > 0 && (!c->step_graph || c->graph_n != n || c->graph_lr != lr)) {
        rc = build_step_graph(c, n, lr);
        if (rc != LBM_OK) return rc;
    }
    cudaError_t e = cudaSuccess;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep)
        e = cudaGraphLaunch(c->step_graph, c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && loss_out) {
        // loss of the parameters after the last update
        forward(c, n);
        backward(c, n);
        e = cudaMemcpyAsync(loss_out, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return fail(e);
}

}  // namespace

extern "C" {

int32_t surr_param_count(void) { return OFF.total; }

int surr_create(uint64_t seed, void* stream, surr_ctx** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    surr_ctx* c = new (std::nothrow) surr_ctx();
    if (!c) return LBM_ERR_NOMEM;
    c->stream = (cudaStream_t)stream;
    const size_t pb = sizeof(float) * OFF.total;
    if (cudaMalloc(&c->params, pb) != cudaSuccess || cudaMalloc(&c->grads, pb) != cudaSuccess ||
        cudaMalloc(&c->m, pb) != cudaSuccess || cudaMalloc(&c->v, pb) != cudaSuccess ||
        cudaMalloc(&c->wq, sizeof(__nv_bfloat16) * OFF.total) != cudaSuccess ||
        cudaMalloc(&c->loss, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->adam_t, sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        surr_destroy(c);
        return LBM_ERR_NOMEM;
    }
    // He initialisation W ~ N(0, 2 / fan_in), b = 0, from a seeded host
    // generator (SplitMix64, Steele, Lea and Flood 2014, and the Box-Muller
    // transform) so that runs are reproducible
    float* host = new (std::nothrow) float[OFF.total];
    if (!host) {
        surr_destroy(c);
        return LBM_ERR_NOMEM;
    }
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uniform = [&]() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    for (int l = 0; l < NLAYER; ++l) {
        const double sd = std::sqrt(2.0 / WIDTH[l]);
        for (int k = 0; k < WIDTH[l + 1] * WIDTH[l]; ++k) {
            const double u1 = uniform(), u2 = uniform();
            host[OFF.w[l] + k] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) *
                                         std::cos(6.283185307179586 * u2));
        }
        for (int k = 0; k < WIDTH[l + 1]; ++k) host[OFF.b[l] + k] = 0.0f;
    }
    const int rc = surr_set_params(c, host);
    delete[] host;
    if (rc != LBM_OK) {
        surr_destroy(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

void surr_destroy(surr_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_batch(c);
    cudaFree(c->params);
    cudaFree(c->grads);
    cudaFree(c->m);
    cudaFree(c->v);
    cudaFree(c->wq);
    cudaFree(c->loss);
    cudaFree(c->adam_t);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

int surr_set_params(surr_ctx* c, const float* params) {
    if (!c || !params) return LBM_ERR_INVALID_ARG;
    const size_t pb = sizeof(float) * OFF.total;
    cudaError_t e = cudaMemcpyAsync(c->params, params, pb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->m, 0, pb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->v, 0, pb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_t, 0, sizeof(long long), c->stream);
    if (e != cudaSuccess) return fail(e);
    refresh_bf16(c);
    return fail(cudaStreamSynchronize(c->stream));
}

int surr_get_params(surr_ctx* c, float* params) {
    if (!c || !params) return LBM_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(params, c->params, sizeof(float) * OFF.total,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return fail(e);
}

int surr_predict(surr_ctx* c, const float* X, int32_t n, float* D_out, float* logit_out) {
    if (!c || !X || n < 1) return LBM_ERR_INVALID_ARG;
    int rc = upload_batch(c, X, nullptr, nullptr, n);
    if (rc != LBM_OK) return rc;
    forward(c, n);
    float* out = new (std::nothrow) float[2 * (size_t)n];
    if (!out) return LBM_ERR_NOMEM;
    cudaError_t e = cudaMemcpyAsync(out, c->act[NLAYER - 1], sizeof(float) * 2 * n,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess)
        for (int s = 0; s < n; ++s) {
            if (D_out) D_out[s] = out[2 * s];
            if (logit_out) logit_out[s] = out[2 * s + 1];
        }
    delete[] out;
    return fail(e);
}

int surr_grad(surr_ctx* c, const float* X, const float* yD, const float* yB, int32_t n,
              float* grads, double* loss) {
    if (!c || !X || !yD || !yB || n < 1) return LBM_ERR_INVALID_ARG;
    int rc = upload_batch(c, X, yD, yB, n);
    if (rc != LBM_OK) return rc;
    forward(c, n);
    backward(c, n);
    cudaError_t e = cudaSuccess;
    if (grads)
        e = cudaMemcpyAsync(grads, c->grads, sizeof(float) * OFF.total, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess && loss)
        e = cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return fail(e);
}

int surr_train(surr_ctx* c, const float* X, const float* yD, const float* yB, int32_t n,
               int32_t epochs, float lr, double* loss_out) {
    if (!c || !X || !yD || !yB || n < 1 || epochs < 0 || !(lr > 0.0f)) return LBM_ERR_INVALID_ARG;
    nvtxRangePushA("surr_train");
    const int rc = train_epochs(c, X, yD, yB, n, epochs, lr, loss_out);
    nvtxRangePop();
    return rc;
}

}  // extern "C"
