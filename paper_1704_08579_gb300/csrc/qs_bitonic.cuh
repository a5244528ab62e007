// Branch-free Bitonic sorting network for sm_103a (Section III-A).
//
// The paper sorts up to 16 AVX-512 vectors with hard-coded permutation
// vectors (Algorithms 1 and 2).  Decoded, its network is the "flip" form of
// Batcher's Bitonic sort in which every comparator puts the minimum at the
// lower index: for each block size s = 2, 4, ..., P the element i is compared
// with its mirror i ^ (s-1) inside the block (Figure 2, "extremities to
// center"), then with i ^ j for j = s/4, ..., 1 (the half-cleaners).
// Algorithm 1's six stages are exactly s=2: xor 1; s=4: xor 3, xor 1;
// s=8: xor 7, xor 2, xor 1.
//
// Here the same network runs on a GPU with the rule-based indexing the paper
// mentions as the alternative to hard-coded tables (Section II-A-3):
//   * element i = t*E + r lives in register r of thread t (blocked layout);
//   * a stage whose partner is in the same thread is a register min/max;
//   * a stage whose partner is in another lane of the warp uses
//     __shfl_xor_sync (the GPU counterpart of the paper's permutexvar);
//   * a stage whose partner is in another warp goes through shared memory.
// Because every comparator sends the minimum to the lower index, padding the
// tail with the largest key (Section III-A-3) never moves: a pad only meets
// elements at lower indices, and a real key never compares greater than the
// largest key.  This also keeps key/value pads from ever swapping with a real
// pair whose key equals the pad.
//
// Key/value (Section III-D): the comparison looks at keys only and the value
// moves with its key.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace qs {

template <class K>
__device__ __forceinline__ bool key_less(K a, K b)
{
    return a < b;
}

// Compare-exchange of two registers of one thread: (a, b) -> (min, max).
template <class K, class V, bool KV>
__device__ __forceinline__ void cmpx(K &a, K &b, V &va, V &vb)
{
    const bool swap = key_less(b, a);
    const K lo = swap ? b : a;
    const K hi = swap ? a : b;
    a = lo;
    b = hi;
    if constexpr (KV) {
        const V vlo = swap ? vb : va;
        const V vhi = swap ? va : vb;
        va = vlo;
        vb = vhi;
    }
}

// Blocked layout inside one warp: E registers per lane, 32*E elements.
// Flip stage of block size s: partner i ^ (s-1).
template <int E, int S, class K, class V, bool KV>
__device__ __forceinline__ void flip_stage_warp(K (&k)[E], V (&v)[E], int lane)
{
    if constexpr (S <= E) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int p = r ^ (S - 1);
            if (r < p) cmpx<K, V, KV>(k[r], k[p], v[r], v[p]);
        }
    } else {
        constexpr int kLaneMask = S / E - 1;  // partner lane = lane ^ kLaneMask
        const bool lower = (lane & (S / E / 2)) == 0;
        K rk[E];
        V rv[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            rk[r] = __shfl_xor_sync(0xffffffffu, k[E - 1 - r], kLaneMask);
            if constexpr (KV) rv[r] = __shfl_xor_sync(0xffffffffu, v[E - 1 - r], kLaneMask);
        }
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const bool take = lower ? key_less(rk[r], k[r]) : key_less(k[r], rk[r]);
            k[r] = take ? rk[r] : k[r];
            if constexpr (KV) v[r] = take ? rv[r] : v[r];
        }
    }
}

// Half-cleaner stage: partner i ^ J.
template <int E, int J, class K, class V, bool KV>
__device__ __forceinline__ void half_stage_warp(K (&k)[E], V (&v)[E], int lane)
{
    if constexpr (J < E) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if ((r & J) == 0) cmpx<K, V, KV>(k[r], k[r | J], v[r], v[r | J]);
        }
    } else {
        constexpr int kLaneMask = J / E;
        const bool lower = (lane & kLaneMask) == 0;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const K o = __shfl_xor_sync(0xffffffffu, k[r], kLaneMask);
            V ov{};
            if constexpr (KV) ov = __shfl_xor_sync(0xffffffffu, v[r], kLaneMask);
            const bool take = lower ? key_less(o, k[r]) : key_less(k[r], o);
            k[r] = take ? o : k[r];
            if constexpr (KV) v[r] = take ? ov : v[r];
        }
    }
}

// Half-cleaners J, J/2, ..., 1 (compile-time recursion keeps indices static).
template <int E, int J, class K, class V, bool KV>
__device__ __forceinline__ void half_cleaners_warp(K (&k)[E], V (&v)[E], int lane)
{
    if constexpr (J >= 1) {
        half_stage_warp<E, J, K, V, KV>(k, v, lane);
        half_cleaners_warp<E, J / 2, K, V, KV>(k, v, lane);
    }
}

// Merge steps for block sizes S, 2S, ..., SMAX, all inside one warp.
template <int E, int S, int SMAX, class K, class V, bool KV>
__device__ __forceinline__ void merges_warp(K (&k)[E], V (&v)[E], int lane)
{
    if constexpr (S <= SMAX) {
        flip_stage_warp<E, S, K, V, KV>(k, v, lane);
        half_cleaners_warp<E, S / 4, K, V, KV>(k, v, lane);
        merges_warp<E, S * 2, SMAX, K, V, KV>(k, v, lane);
    }
}

// Sorts the 32*E elements held by one warp (blocked layout).
template <int E, class K, class V, bool KV>
__device__ __forceinline__ void warp_bitonic_sort(K (&k)[E], V (&v)[E])
{
    merges_warp<E, 2, 32 * E, K, V, KV>(k, v, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// CTA-wide network: NT threads x E registers = P elements.  Stages whose
// partner lies in another warp run in shared memory, padded by one element
// every 32 to keep the blocked write/read free of bank conflicts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

template <int NT, int E, class K, class V, bool KV>
__device__ __forceinline__ void regs_to_smem(const K (&k)[E], const V (&v)[E], K *sk, V *sv)
{
    const int base = threadIdx.x * E;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        sk[pad32(base + r)] = k[r];
        if constexpr (KV) sv[pad32(base + r)] = v[r];
    }
}

template <int NT, int E, class K, class V, bool KV>
__device__ __forceinline__ void smem_to_regs(K (&k)[E], V (&v)[E], const K *sk, const V *sv)
{
    const int base = threadIdx.x * E;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        k[r] = sk[pad32(base + r)];
        if constexpr (KV) v[r] = sv[pad32(base + r)];
    }
}

template <class K, class V, bool KV>
__device__ __forceinline__ void smem_cmpx(K *sk, V *sv, int lo, int hi)
{
    const int a = pad32(lo), b = pad32(hi);
    K ka = sk[a], kb = sk[b];
    if (key_less(kb, ka)) {
        sk[a] = kb;
        sk[b] = ka;
        if constexpr (KV) {
            V t = sv[a];
            sv[a] = sv[b];
            sv[b] = t;
        }
    }
}

// One flip stage (block size s) over P elements in shared memory.
template <int NT, int P, class K, class V, bool KV>
__device__ __forceinline__ void smem_flip(K *sk, V *sv, int s)
{
    const int half = s >> 1;
    for (int c = threadIdx.x; c < P / 2; c += NT) {
        const int blk = c / half, w = c - blk * half;
        smem_cmpx<K, V, KV>(sk, sv, blk * s + w, blk * s + s - 1 - w);
    }
}

template <int NT, int P, class K, class V, bool KV>
__device__ __forceinline__ void smem_half(K *sk, V *sv, int j)
{
    for (int c = threadIdx.x; c < P / 2; c += NT) {
        const int blk = c / j, w = c - blk * j;
        const int lo = blk * 2 * j + w;
        smem_cmpx<K, V, KV>(sk, sv, lo, lo + j);
    }
}

template <int NT, int E, int S, class K, class V, bool KV>
__device__ __forceinline__ void merges_cta(K (&k)[E], V (&v)[E], K *sk, V *sv)
{
    constexpr int P = NT * E;
    if constexpr (S <= P) {
        const int lane = threadIdx.x & 31;
        if constexpr (S <= 32 * E) {
            flip_stage_warp<E, S, K, V, KV>(k, v, lane);
            half_cleaners_warp<E, S / 4, K, V, KV>(k, v, lane);
        } else {
            regs_to_smem<NT, E, K, V, KV>(k, v, sk, sv);
            __syncthreads();
            smem_flip<NT, P, K, V, KV>(sk, sv, S);
            __syncthreads();
            for (int j = S / 4; j >= 32 * E; j >>= 1) {
                smem_half<NT, P, K, V, KV>(sk, sv, j);
                __syncthreads();
            }
            smem_to_regs<NT, E, K, V, KV>(k, v, sk, sv);
            __syncthreads();
            half_cleaners_warp<E, 16 * E, K, V, KV>(k, v, lane);
        }
        merges_cta<NT, E, S * 2, K, V, KV>(k, v, sk, sv);
    }
}

// Sorts NT*E elements held by the CTA (blocked layout); sk/sv hold at least
// pad32(NT*E) elements.
template <int NT, int E, class K, class V, bool KV>
__device__ __forceinline__ void cta_bitonic_sort(K (&k)[E], V (&v)[E], K *sk, V *sv)
{
    merges_cta<NT, E, 2, K, V, KV>(k, v, sk, sv);
}

}  // namespace qs
