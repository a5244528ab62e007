// Splitter MLP for the learned form of the sort (a growth line of the method;
// the paper has no model).  FP32, hand-written SIMT kernels: the network is
// tiny (86,400 parameters, one sketch per array at inference), so it is a
// latency problem, not a dense-contraction throughput problem.
//
//   x (1024-key sorted sample, min-max scaled to [0,1])
//   -> h1 = relu(W1 x + b1) (64) -> h2 = relu(W2 h1 + b2) (64)
//   -> z = W3 h2 + b3 (256) -> d = softplus(z) -> c = cumsum(d)
//   -> q_j = c_j / c_255, j = 0..254: monotone quantile estimates in [0, 1].
// Parameters: one flat float array W1 (64x1024 row-major), b1, W2 (64x64), b2,
// W3 (256x64), b3.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qs_internal.h"

namespace qs {
namespace mlp {

constexpr int kIn = 1024, kHid = 64, kOut = 256, kSplit = 255;
constexpr int kW1 = 0, kB1 = kW1 + kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
              kB3 = kW3 + kOut * kHid, kNParams = kB3 + kOut;
// Saved activations per sample: a1 (64), a2 (64), z (256), c (256).
constexpr int kActA1 = 0, kActA2 = 64, kActZ = 128, kActC = 384, kAct = 640;
// Per-sample backward vectors: gz (256), ga2 (64), ga1 (64).
constexpr int kWGz = 0, kWGa2 = 256, kWGa1 = 320, kWork = 384;
constexpr int kNT = 256;  // threads per CTA

struct Smem {
    float x[kIn];
    float a1[kHid], h1[kHid], a2[kHid], h2[kHid];
    float z[kOut], c[kOut];
    float wsum[kNT / 32];
    float g[kOut];
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float softplusf(float z) { return z > 20.f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigmoidf(float z) { return 1.f / (1.f + expf(-z)); }

// Inclusive scan of s[0..255] in place (256 threads); reverse = suffix sums.
__device__ __forceinline__ void cta_scan256(float *s, Smem &sm, bool reverse)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int idx = reverse ? kOut - 1 - t : t;
    float v = s[idx];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) sm.wsum[w] = v;
    __syncthreads();
    float add = 0.f;
    for (int i = 0; i < w; ++i) add += sm.wsum[i];
    __syncthreads();
    s[idx] = v + add;
    __syncthreads();
}

// Forward pass of one sample held in sm.x (whole CTA).  Leaves a1, h1, a2, h2,
// z, c in shared memory.
static __device__ void forward_cta(const float *__restrict__ P, Smem &sm)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int o = w; o < kHid; o += kNT / 32) {  // layer 1: one warp per output
        const float *row = P + kW1 + o * kIn;
        float acc = 0.f;
        for (int i = lane; i < kIn; i += 32) acc += row[i] * sm.x[i];
        acc = warp_sum(acc);
        if (lane == 0) {
            const float a = acc + P[kB1 + o];
            sm.a1[o] = a;
            sm.h1[o] = a > 0.f ? a : 0.f;
        }
    }
    __syncthreads();
    for (int o = w; o < kHid; o += kNT / 32) {  // layer 2
        const float *row = P + kW2 + o * kHid;
        float acc = row[lane] * sm.h1[lane] + row[lane + 32] * sm.h1[lane + 32];
        acc = warp_sum(acc);
        if (lane == 0) {
            const float a = acc + P[kB2 + o];
            sm.a2[o] = a;
            sm.h2[o] = a > 0.f ? a : 0.f;
        }
    }
    __syncthreads();
    for (int o = w; o < kOut; o += kNT / 32) {  // layer 3
        const float *row = P + kW3 + o * kHid;
        float acc = row[lane] * sm.h2[lane] + row[lane + 32] * sm.h2[lane + 32];
        acc = warp_sum(acc);
        if (lane == 0) sm.z[o] = acc + P[kB3 + o];
    }
    __syncthreads();
    sm.c[t] = softplusf(sm.z[t]);
    __syncthreads();
    cta_scan256(sm.c, sm, false);
}

}  // namespace mlp
}  // namespace qs
