// Host launchers of the splitter-MLP kernels (kind-independent).
#include <cmath>

#include "qs_mlp.cuh"

namespace qs {
namespace mlp {

// q[b][j] = c_j / c_255 for every sample b; saves activations for backward.
__global__ void __launch_bounds__(kNT) forward_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                                      float *__restrict__ Q, float *__restrict__ ACT)
{
    __shared__ Smem sm;
    const int b = blockIdx.x, t = threadIdx.x;
    for (int i = t; i < kIn; i += kNT) sm.x[i] = X[static_cast<int64_t>(b) * kIn + i];
    __syncthreads();
    forward_cta(P, sm);
    const float S = sm.c[kOut - 1];
    if (t < kSplit) Q[static_cast<int64_t>(b) * kSplit + t] = sm.c[t] / S;
    if (ACT) {
        float *act = ACT + static_cast<int64_t>(b) * kAct;
        if (t < kHid) {
            act[kActA1 + t] = sm.a1[t];
            act[kActA2 + t] = sm.a2[t];
        }
        act[kActZ + t] = sm.z[t];
        act[kActC + t] = sm.c[t];
    }
}

// Backward, part 1: per-sample output-side vectors gz, ga2, ga1 and the loss
// (mean over batch x 255 of (q - t)^2), by the chain rule through the
// normalisation, the cumulative sum, softplus and the two ReLU layers.
__global__ void __launch_bounds__(kNT) backward_vec_kernel(const float *__restrict__ P, const float *__restrict__ T,
                                                           const float *__restrict__ ACT, int64_t batch,
                                                           float *__restrict__ WORK, float *__restrict__ loss)
{
    __shared__ Smem sm;
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const float *act = ACT + static_cast<int64_t>(b) * kAct;
    const float *tb = T + static_cast<int64_t>(b) * kSplit;
    if (t < kHid) {
        sm.a1[t] = act[kActA1 + t];
        sm.a2[t] = act[kActA2 + t];
    }
    sm.z[t] = act[kActZ + t];
    sm.c[t] = act[kActC + t];
    __syncthreads();
    const float scale = 1.f / (static_cast<float>(batch) * kSplit);
    const float S = sm.c[kOut - 1];
    float gq = 0.f, contrib = 0.f, l = 0.f;
    if (t < kSplit) {
        const float e = sm.c[t] / S - tb[t];
        l = e * e * scale;
        gq = 2.f * e * scale;
        contrib = gq * sm.c[t];
    }
    // sum of gq_j c_j and of the loss over the CTA
    float r1 = warp_sum(contrib), r2 = warp_sum(l);
    if (lane == 0) sm.wsum[w] = r1;
    __syncthreads();
    float tail = 0.f;
    for (int i = 0; i < kNT / 32; ++i) tail += sm.wsum[i];
    __syncthreads();
    if (lane == 0 && loss) atomicAdd(loss, r2);
    // gc_k = gq_k / S (k < 255); gc_255 = -sum_j gq_j c_j / S^2
    sm.g[t] = t < kSplit ? gq / S : -tail / (S * S);
    __syncthreads();
    cta_scan256(sm.g, sm, true);  // gd_i = sum_{k >= i} gc_k
    const float gz = sm.g[t] * sigmoidf(sm.z[t]);
    sm.g[t] = gz;
    WORK[static_cast<int64_t>(b) * kWork + kWGz + t] = gz;
    __syncthreads();
    // gh2 = W3^T gz; ga2 = gh2 * [a2 > 0]
    for (int i = w; i < kHid; i += kNT / 32) {
        float acc = 0.f;
        for (int o = lane; o < kOut; o += 32) acc += P[kW3 + o * kHid + i] * sm.g[o];
        acc = warp_sum(acc);
        if (lane == 0) sm.h2[i] = sm.a2[i] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // gh1 = W2^T ga2; ga1 = gh1 * [a1 > 0]
    for (int i = w; i < kHid; i += kNT / 32) {
        float acc = P[kW2 + lane * kHid + i] * sm.h2[lane] + P[kW2 + (lane + 32) * kHid + i] * sm.h2[lane + 32];
        acc = warp_sum(acc);
        if (lane == 0) sm.h1[i] = sm.a1[i] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    if (t < kHid) {
        WORK[static_cast<int64_t>(b) * kWork + kWGa2 + t] = sm.h2[t];
        WORK[static_cast<int64_t>(b) * kWork + kWGa1 + t] = sm.h1[t];
    }
}

// Backward, part 2: every parameter's gradient as a sum over the batch (one
// thread per parameter; no atomics, so the result is deterministic).
__global__ void backward_param_kernel(const float *__restrict__ X, const float *__restrict__ ACT,
                                      const float *__restrict__ WORK, int64_t batch, float *__restrict__ G)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNParams) return;
    float acc = 0.f;
    if (p < kB1) {  // W1[o][i]: ga1[o] * x[i]
        const int o = p / kIn, i = p - o * kIn;
        for (int64_t b = 0; b < batch; ++b) acc += WORK[b * kWork + kWGa1 + o] * X[b * kIn + i];
    } else if (p < kW2) {
        const int o = p - kB1;
        for (int64_t b = 0; b < batch; ++b) acc += WORK[b * kWork + kWGa1 + o];
    } else if (p < kB2) {  // W2[o][i]: ga2[o] * h1[i]
        const int q = p - kW2, o = q / kHid, i = q - o * kHid;
        for (int64_t b = 0; b < batch; ++b) {
            const float a1 = ACT[b * kAct + kActA1 + i];
            acc += WORK[b * kWork + kWGa2 + o] * (a1 > 0.f ? a1 : 0.f);
        }
    } else if (p < kW3) {
        const int o = p - kB2;
        for (int64_t b = 0; b < batch; ++b) acc += WORK[b * kWork + kWGa2 + o];
    } else if (p < kB3) {  // W3[o][i]: gz[o] * h2[i]
        const int q = p - kW3, o = q / kHid, i = q - o * kHid;
        for (int64_t b = 0; b < batch; ++b) {
            const float a2 = ACT[b * kAct + kActA2 + i];
            acc += WORK[b * kWork + kWGz + o] * (a2 > 0.f ? a2 : 0.f);
        }
    } else {
        const int o = p - kB3;
        for (int64_t b = 0; b < batch; ++b) acc += WORK[b * kWork + kWGz + o];
    }
    G[p] = acc;
}

// Adam (Kingma & Ba 2015) with bias correction; step counts from 1.  The
// decay weights and both (1 - beta) factors come from the host, computed in
// double: 1 - 0.999f alone would be off by 1.3e-5 relative.
__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, float lr, float b1, float omb1, float b2, float omb2, float eps,
                            float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNParams) return;
    const float g = G[p];
    const float m = b1 * M[p] + omb1 * g;
    const float v = b2 * V[p] + omb2 * g * g;
    M[p] = m;
    V[p] = v;
    P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace mlp

int mlp_param_count() { return mlp::kNParams; }

int mlp_forward(const float *P, const float *X, int64_t batch, float *Q, float *ACT, void *stream)
{
    if (batch <= 0) return cudaSuccess;
    mlp::forward_kernel<<<static_cast<unsigned>(batch), mlp::kNT, 0, static_cast<cudaStream_t>(stream)>>>(P, X, Q, ACT);
    return static_cast<int>(cudaGetLastError());
}

int mlp_backward(const float *P, const float *X, const float *T, const float *ACT, int64_t batch, float *WORK, float *G,
                 float *loss, void *stream)
{
    if (batch <= 0) return cudaSuccess;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (loss) cudaMemsetAsync(loss, 0, sizeof(float), s);
    mlp::backward_vec_kernel<<<static_cast<unsigned>(batch), mlp::kNT, 0, s>>>(P, T, ACT, batch, WORK, loss);
    mlp::backward_param_kernel<<<(mlp::kNParams + 255) / 256, 256, 0, s>>>(X, ACT, WORK, batch, G);
    return static_cast<int>(cudaGetLastError());
}

int mlp_adam(float *P, const float *G, float *M, float *V, int64_t step, float lr, void *stream)
{
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    const double c1 = 1.0 - std::pow(b1, static_cast<double>(step));
    const double c2 = 1.0 - std::pow(b2, static_cast<double>(step));
    mlp::adam_kernel<<<(mlp::kNParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        P, G, M, V, lr, static_cast<float>(b1), static_cast<float>(1.0 - b1), static_cast<float>(b2),
        static_cast<float>(1.0 - b2), static_cast<float>(eps), static_cast<float>(c1), static_cast<float>(c2));
    return static_cast<int>(cudaGetLastError());
}

}  // namespace qs
