// Schedule cost model: forward, backward and Adam kernels of a small FP32
// MLP (NTT_MLP_IN -> 64 -> 64 -> NTT_MLP_OUT, ReLU) that predicts the
// log-time of every candidate schedule of a transform shape.  The switch
// point and fused-stage choice of Sec. V-D are decided here by a model
// trained on measured timings instead of a closed-form rule.
//
// Parameter vector (float, NTT_MLP_PARAMS entries, row-major):
//   W1[64][IN], b1[64], W2[64][64], b2[64], W3[OUT][64], b3[OUT]
// Activations per sample (NTT_MLP_ACTS floats): h1[64], h2[64], y[OUT]
// (h = ReLU(W x + b) after each hidden layer; y is linear).
// Loss: masked mean squared error over the valid outputs,
//   L = sum_{b,k} m[b,k] (y[b,k] - t[b,k])^2 / sum_{b,k} m[b,k].
// Gradient sums over the batch are plain per-parameter loops (no atomics),
// so the gradients are deterministic.
#include <cuda_runtime.h>

#include "ntt_gb300.h"

namespace nttgb {

constexpr int IN = NTT_MLP_IN, H = NTT_MLP_HIDDEN, OUT = NTT_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + OUT * H, N_PARAMS = OFF_B3 + OUT;
static_assert(N_PARAMS == NTT_MLP_PARAMS, "parameter layout");
constexpr int A_H1 = 0, A_H2 = H, A_Y = 2 * H, N_ACT = 2 * H + OUT;
static_assert(N_ACT == NTT_MLP_ACTS, "activation layout");

// y[b][o] = act(bias[o] + sum_i x[b][i] W[o][i]); one thread per (b, o)
__global__ void k_dense_fwd(const float* __restrict__ x, int x_stride, const float* __restrict__ W,
                            const float* __restrict__ bias, float* y, int y_stride, int n_in, int n_out,
                            uint32_t batch, int relu) {
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (uint64_t)batch * n_out) return;
    const uint32_t b = (uint32_t)(idx / n_out);
    const int o = (int)(idx % n_out);
    float acc = bias[o];
    const float* xr = x + (uint64_t)b * x_stride;
    const float* wr = W + (uint64_t)o * n_in;
    for (int i = 0; i < n_in; ++i) acc = fmaf(xr[i], wr[i], acc);
    y[(uint64_t)b * y_stride + o] = relu ? fmaxf(acc, 0.0f) : acc;
}

// dY of the masked MSE, and the per-sample sums of the loss terms
__global__ void k_mse_grad(const float* __restrict__ act, const float* __restrict__ target,
                           const float* __restrict__ mask, uint32_t batch, float inv_count, float* dz,
                           float* loss_terms) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    float s = 0.0f;
    for (int k = 0; k < OUT; ++k) {
        const float m = mask[(uint64_t)b * OUT + k];
        const float d = act[(uint64_t)b * N_ACT + A_Y + k] - target[(uint64_t)b * OUT + k];
        dz[(uint64_t)b * N_ACT + A_Y + k] = 2.0f * m * d * inv_count;
        s += m * d * d;
    }
    loss_terms[b] = s * inv_count;
}

// dW[o][i] = sum_b dz[b][o] x[b][i];  db[o] = sum_b dz[b][o]  (thread per weight)
__global__ void k_dense_bwd_w(const float* __restrict__ x, int x_stride, const float* __restrict__ dz,
                              int dz_stride, int n_in, int n_out, uint32_t batch, float* dW, float* db) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_out * (n_in + 1)) return;
    const int o = idx / (n_in + 1), i = idx % (n_in + 1);
    float acc = 0.0f;
    if (i < n_in) {
        for (uint32_t b = 0; b < batch; ++b)
            acc = fmaf(dz[(uint64_t)b * dz_stride + o], x[(uint64_t)b * x_stride + i], acc);
        dW[(uint64_t)o * n_in + i] = acc;
    } else {
        for (uint32_t b = 0; b < batch; ++b) acc += dz[(uint64_t)b * dz_stride + o];
        db[o] = acc;
    }
}

// dz_prev[b][i] = (sum_o dz[b][o] W[o][i]) * [h_prev[b][i] > 0]   (ReLU of the layer below)
__global__ void k_dense_bwd_x(const float* __restrict__ dz, int dz_stride, const float* __restrict__ W,
                              const float* __restrict__ h_prev, int h_stride, float* dz_prev, int dzp_stride,
                              int n_in, int n_out, uint32_t batch) {
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (uint64_t)batch * n_in) return;
    const uint32_t b = (uint32_t)(idx / n_in);
    const int i = (int)(idx % n_in);
    float acc = 0.0f;
    for (int o = 0; o < n_out; ++o) acc = fmaf(dz[(uint64_t)b * dz_stride + o], W[(uint64_t)o * n_in + i], acc);
    dz_prev[(uint64_t)b * dzp_stride + i] = h_prev[(uint64_t)b * h_stride + i] > 0.0f ? acc : 0.0f;
}

__global__ void k_sum(const float* __restrict__ v, uint32_t n, float* out) {
    __shared__ float s[256];
    float acc = 0.0f;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_adam(float* p, const float* __restrict__ g, float* m, float* v, uint32_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static unsigned blocks_for(uint64_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

}  // namespace nttgb

using namespace nttgb;

extern "C" {

int ntt_mlp_forward(const float* d_params, const float* d_x, uint32_t batch, float* d_act, void* cuda_stream) {
    if (!d_params || !d_x || !d_act || batch == 0) return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float* P = d_params;
    k_dense_fwd<<<blocks_for((uint64_t)batch * H, 256), 256, 0, st>>>(d_x, IN, P + OFF_W1, P + OFF_B1,
                                                                       d_act + A_H1, N_ACT, IN, H, batch, 1);
    k_dense_fwd<<<blocks_for((uint64_t)batch * H, 256), 256, 0, st>>>(d_act + A_H1, N_ACT, P + OFF_W2,
                                                                       P + OFF_B2, d_act + A_H2, N_ACT, H, H,
                                                                       batch, 1);
    k_dense_fwd<<<blocks_for((uint64_t)batch * OUT, 256), 256, 0, st>>>(d_act + A_H2, N_ACT, P + OFF_W3,
                                                                         P + OFF_B3, d_act + A_Y, N_ACT, H,
                                                                         OUT, batch, 0);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

int ntt_mlp_backward(const float* d_params, const float* d_x, const float* d_act, const float* d_target,
                     const float* d_mask, uint32_t batch, float mask_count, float* d_grad, float* d_work,
                     float* d_loss, void* cuda_stream) {
    if (!d_params || !d_x || !d_act || !d_target || !d_mask || !d_grad || !d_work || batch == 0 ||
        !(mask_count > 0.0f))
        return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float* P = d_params;
    float* G = d_grad;
    float* dz = d_work;                               // [batch][N_ACT]: dz of h1, h2, y
    float* loss_terms = d_work + (uint64_t)batch * N_ACT;   // [batch]
    k_mse_grad<<<blocks_for(batch, 256), 256, 0, st>>>(d_act, d_target, d_mask, batch, 1.0f / mask_count, dz,
                                                       loss_terms);
    // layer 3 (linear): dW3, db3, then dz of h2
    k_dense_bwd_w<<<blocks_for(OUT * (H + 1), 256), 256, 0, st>>>(d_act + A_H2, N_ACT, dz + A_Y, N_ACT, H, OUT,
                                                                  batch, G + OFF_W3, G + OFF_B3);
    k_dense_bwd_x<<<blocks_for((uint64_t)batch * H, 256), 256, 0, st>>>(dz + A_Y, N_ACT, P + OFF_W3,
                                                                         d_act + A_H2, N_ACT, dz + A_H2, N_ACT,
                                                                         H, OUT, batch);
    // layer 2
    k_dense_bwd_w<<<blocks_for(H * (H + 1), 256), 256, 0, st>>>(d_act + A_H1, N_ACT, dz + A_H2, N_ACT, H, H,
                                                                batch, G + OFF_W2, G + OFF_B2);
    k_dense_bwd_x<<<blocks_for((uint64_t)batch * H, 256), 256, 0, st>>>(dz + A_H2, N_ACT, P + OFF_W2,
                                                                         d_act + A_H1, N_ACT, dz + A_H1, N_ACT,
                                                                         H, H, batch);
    // layer 1
    k_dense_bwd_w<<<blocks_for(H * (IN + 1), 256), 256, 0, st>>>(d_x, IN, dz + A_H1, N_ACT, IN, H, batch,
                                                                 G + OFF_W1, G + OFF_B1);
    if (d_loss) k_sum<<<1, 256, 0, st>>>(loss_terms, batch, d_loss);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

int ntt_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, uint32_t n, float lr,
                 float beta1, float beta2, float eps, uint32_t step, void* cuda_stream) {
    if (!d_params || !d_grad || !d_m || !d_v || n == 0 || step == 0) return NTT_ERR_ARG;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<blocks_for(n, 256), 256, 0, (cudaStream_t)cuda_stream>>>(d_params, d_grad, d_m, d_v, n, lr, beta1,
                                                                       beta2, eps, c1, c2);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // extern "C"
