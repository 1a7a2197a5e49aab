// k_mlp.cu -- the learned early-stop model (a project addition; the paper's
// search has no learned part): a 2-layer perceptron, 8 inputs -> 64 ReLU
// hidden units -> 1 logit, trained on traces of the plain search.
//
// Parameters are one flat f32 vector of NHQ_MLP_PARAMS values,
//   W1 [8][64] (input-major) | b1 [64] | W2 [64] | b2,
// the master copy for training.  Inference (in the search kernel and in
// nhq_mlp_forward) reads an fp16 copy and accumulates in f32.
//
// Training: mean binary cross-entropy with logits; one thread per sample runs
// the forward pass, the loss gradient and the backward pass, each gradient
// entry is summed over the warp with shuffles and added to global memory by
// lane 0; an Adam step updates the master weights.
#include <cmath>
#include <vector>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr int kIn = NHQ_MLP_INPUTS, kHid = NHQ_MLP_HIDDEN, kParams = NHQ_MLP_PARAMS;
constexpr int oW1 = 0, oB1 = kIn * kHid, oW2 = oB1 + kHid, oB2 = oW2 + kHid;
constexpr unsigned FULL = 0xFFFFFFFFu;

__global__ void to_half_kernel(const float *__restrict__ p, __half *__restrict__ h, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        h[i] = __float2half_rn(p[i]);
}

// one warp per sample: the same arithmetic as the search kernel's decision
__global__ void mlp_forward_kernel(const __half *__restrict__ w, const float *__restrict__ X,
                                   int64_t n, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n)
        return;
    float f[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i)
        f[i] = X[s * kIn + i];
    const float logit = mlp_logit_warp(w, f, lane);
    if (lane == 0)
        out[s] = logit;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// gradient of the mean loss over `total` samples, accumulated into g[kParams] and *loss
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float *__restrict__ params,
                                                       const float *__restrict__ X,
                                                       const float *__restrict__ y, int64_t n,
                                                       float inv_total, float *__restrict__ g,
                                                       float *__restrict__ loss) {
    __shared__ float w[kParams];
    for (int i = threadIdx.x; i < kParams; i += blockDim.x)
        w[i] = params[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s < n;
    float x[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i)
        x[i] = live ? X[s * kIn + i] : 0.f;
    const float yy = live ? y[s] : 0.f;
    float sc = w[oB2];
    for (int j = 0; j < kHid; ++j) {
        float z = w[oB1 + j];
#pragma unroll
        for (int i = 0; i < kIn; ++i)
            z = fmaf(w[oW1 + i * kHid + j], x[i], z);
        sc = fmaf(w[oW2 + j], fmaxf(z, 0.f), sc);
    }
    const float p = 1.f / (1.f + expf(-sc));
    const float ds = live ? (p - yy) * inv_total : 0.f;
    const float l = live ? (fmaxf(sc, 0.f) + log1pf(expf(-fabsf(sc))) - yy * sc) * inv_total : 0.f;
    for (int j = 0; j < kHid; ++j) {
        float z = w[oB1 + j];
#pragma unroll
        for (int i = 0; i < kIn; ++i)
            z = fmaf(w[oW1 + i * kHid + j], x[i], z);
        const float h = fmaxf(z, 0.f);
        const float dz = z > 0.f ? ds * w[oW2 + j] : 0.f;
        const float gw2 = warp_sum(ds * h);
        const float gb1 = warp_sum(dz);
        if (lane == 0) {
            atomicAdd(&g[oW2 + j], gw2);
            atomicAdd(&g[oB1 + j], gb1);
        }
#pragma unroll
        for (int i = 0; i < kIn; ++i) {
            const float gw1 = warp_sum(dz * x[i]);
            if (lane == 0)
                atomicAdd(&g[oW1 + i * kHid + j], gw1);
        }
    }
    const float gb2 = warp_sum(ds), ls = warp_sum(l);
    if (lane == 0) {
        atomicAdd(&g[oB2], gb2);
        atomicAdd(loss, ls);
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int n, float lr,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m[i] = b1 * m[i] + (1.f - b1) * g[i];
    v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] * c1) / (sqrtf(v[i] * c2) + eps);
}

// trace labels: stopping at a traced expansion returns the final top-k
__global__ void label_kernel(const unsigned long long *__restrict__ h,
                             const int32_t *__restrict__ tq,
                             const unsigned long long *__restrict__ fin, int64_t n,
                             uint8_t *__restrict__ lab) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        lab[i] = h[i] == fin[tq[i]] ? 1 : 0;
}

thread_local void *g_mlp_scratch = nullptr;
thread_local size_t g_mlp_scratch_bytes = 0;

cudaError_t mlp_scratch(size_t need, void **out) {
    if (g_mlp_scratch_bytes < need) {
        if (g_mlp_scratch) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess)
                return e;
            cudaFree(g_mlp_scratch);
            g_mlp_scratch = nullptr;
            g_mlp_scratch_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&g_mlp_scratch, need);
        if (e != cudaSuccess)
            return e;
        g_mlp_scratch_bytes = need;
    }
    *out = g_mlp_scratch;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_mlp_to_half(const float *params, __half *w16, cudaStream_t s) {
    to_half_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(params, w16, kParams);
    return cudaGetLastError();
}

cudaError_t launch_trace_labels(const unsigned long long *hash, const int32_t *tq,
                                const unsigned long long *final_hash, int64_t n, uint8_t *lab,
                                cudaStream_t s) {
    if (n <= 0)
        return cudaSuccess;
    label_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(hash, tq, final_hash, n, lab);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const float *params, const float *X, int64_t n, float *logits,
                        cudaStream_t s) {
    void *sc = nullptr;
    cudaError_t e = mlp_scratch(sizeof(__half) * kParams, &sc);
    if (e != cudaSuccess)
        return e;
    __half *w16 = reinterpret_cast<__half *>(sc);
    if ((e = launch_mlp_to_half(params, w16, s)) != cudaSuccess)
        return e;
    if (n <= 0)
        return cudaSuccess;
    mlp_forward_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(w16, X, n, logits);
    return cudaGetLastError();
}

cudaError_t mlp_grad(const float *params, const float *X, const float *y, int64_t n,
                     int64_t total, float *g, float *loss, cudaStream_t s) {
    if (n <= 0)
        return cudaSuccess;
    mlp_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, X, y, n,
                                                                 1.f / (float)total, g, loss);
    return cudaGetLastError();
}

cudaError_t mlp_train(float *params, const float *X, const float *y, int64_t n, int epochs,
                      int batch, float lr, cudaStream_t s) {
    void *sc = nullptr;
    cudaError_t e = mlp_scratch(sizeof(float) * (3 * kParams + 1), &sc);
    if (e != cudaSuccess)
        return e;
    float *g = reinterpret_cast<float *>(sc), *m = g + kParams, *v = m + kParams,
          *loss = v + kParams;
    if ((e = cudaMemsetAsync(m, 0, sizeof(float) * 2 * kParams, s)) != cudaSuccess)
        return e;
    int t = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t b = 0; b < n; b += batch) {
            const int64_t nb = n - b < batch ? n - b : batch;
            if ((e = cudaMemsetAsync(g, 0, sizeof(float) * (kParams + 1), s)) != cudaSuccess)
                return e;
            if ((e = mlp_grad(params, X + b * kIn, y + b, nb, nb, g, loss, s)) != cudaSuccess)
                return e;
            ++t;
            const float c1 = 1.f / (1.f - powf(0.9f, (float)t));
            const float c2 = 1.f / (1.f - powf(0.999f, (float)t));
            adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(params, g, m, v, kParams, lr, c1,
                                                              c2);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

}  // namespace nhq
