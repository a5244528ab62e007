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
// Here the same network runs with the rule-based indexing the paper mentions
// as the alternative to hard-coded tables (Section II-A-3):
//   * element i = t*E + r lives in register r of thread t (blocked layout);
//   * a stage whose partner is in the same thread is a register min/max,
//     generated at compile time (it does not depend on the block size);
//   * a stage whose partner is in another lane of the warp uses
//     __shfl_xor_sync (the GPU counterpart of the paper's permutexvar), in a
//     run-time loop over block sizes so the code stays small;
//   * a stage whose partner is in another warp runs in shared memory.
// Because every comparator sends the minimum to the lower index, padding the
// tail with the largest key (Section III-A-3) never moves: a pad only meets
// elements at lower indices, and no key compares greater than the largest
// key.  Keys are compared as integers ("sort space"); key/value pairs are
// packed into one 64-bit word with the key in the high half (Section III-D:
// the value moves with its key).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace qs {

// (a, b) -> (min, max); equal keys stay put.
template <class S>
__device__ __forceinline__ void cx(S &a, S &b)
{
    const bool sw = b < a;
    const S lo = sw ? b : a;
    b = sw ? a : b;
    a = lo;
}

// Half-cleaners J, J/2, ..., 1 inside one thread's registers.
template <int E, int J, class S>
__device__ __forceinline__ void reg_half(S (&k)[E])
{
    if constexpr (J >= 1) {
#pragma unroll
        for (int r = 0; r < E; ++r)
            if ((r & J) == 0) cx(k[r], k[r | J]);
        reg_half<E, J / 2>(k);
    }
}

// Merge steps for block sizes SZ, 2*SZ, ..., E inside one thread.
template <int E, int SZ, class S>
__device__ __forceinline__ void reg_merges(S (&k)[E])
{
    if constexpr (SZ <= E) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int p = r ^ (SZ - 1);
            if (r < p) cx(k[r], k[p]);
        }
        reg_half<E, SZ / 4>(k);
        reg_merges<E, SZ * 2, S>(k);
    }
}

// Flip stage across lanes: lane l pairs with l ^ lm, register r with E-1-r.
// `upper` is true on the lane holding the higher indices (keeps the maximum).
template <int E, class S>
__device__ __forceinline__ void shfl_flip(S (&k)[E], int lm, bool upper)
{
    S o[E];
#pragma unroll
    for (int r = 0; r < E; ++r) o[r] = __shfl_xor_sync(0xffffffffu, k[E - 1 - r], lm);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const bool take = upper ? (k[r] < o[r]) : (o[r] < k[r]);
        k[r] = take ? o[r] : k[r];
    }
}

// Half-cleaner across lanes: lane l pairs with l ^ m, same register.
template <int E, class S>
__device__ __forceinline__ void shfl_half(S (&k)[E], int m, bool upper)
{
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const S o = __shfl_xor_sync(0xffffffffu, k[r], m);
        const bool take = upper ? (k[r] < o) : (o < k[r]);
        k[r] = take ? o : k[r];
    }
}

// Sorts the 32*E elements held by one warp (blocked layout).
template <int E, class S>
__device__ __forceinline__ void warp_bitonic_sort(S (&k)[E])
{
    const int lane = threadIdx.x & 31;
    reg_merges<E, 2, S>(k);
    for (int sz = 2 * E; sz <= 32 * E; sz <<= 1) {
        shfl_flip<E, S>(k, sz / E - 1, (lane & (sz / E / 2)) != 0);
        for (int j = sz / 4; j >= E; j >>= 1) shfl_half<E, S>(k, j / E, (lane & (j / E)) != 0);
        reg_half<E, E / 2>(k);
    }
}

// ---------------------------------------------------------------------------
// CTA-wide network: NT threads x E registers = P elements.  Stages whose
// partner lies in another warp run in shared memory, padded by one element
// every 32 to keep the blocked write/read free of bank conflicts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

template <int E, class S>
__device__ __forceinline__ void regs_to_smem(const S (&k)[E], S *sk)
{
    const int base = threadIdx.x * E;
#pragma unroll
    for (int r = 0; r < E; ++r) sk[pad32(base + r)] = k[r];
}

template <int E, class S>
__device__ __forceinline__ void smem_to_regs(S (&k)[E], const S *sk)
{
    const int base = threadIdx.x * E;
#pragma unroll
    for (int r = 0; r < E; ++r) k[r] = sk[pad32(base + r)];
}

template <class S>
__device__ __forceinline__ void smem_cx(S *sk, int lo, int hi)
{
    const int a = pad32(lo), b = pad32(hi);
    S x = sk[a], y = sk[b];
    cx(x, y);
    sk[a] = x;
    sk[b] = y;
}

// Flip stage of block size 2^(lh+1) over P elements in shared memory.
template <int NT, int P, class S>
__device__ __forceinline__ void smem_flip(S *sk, int lh)
{
    const int half = 1 << lh;
#pragma unroll 4
    for (int c = threadIdx.x; c < P / 2; c += NT) {
        const int blk = c >> lh, w = c & (half - 1);
        const int b0 = blk << (lh + 1);
        smem_cx(sk, b0 + w, b0 + 2 * half - 1 - w);
    }
}

// Half-cleaner with partner distance 2^lj.
template <int NT, int P, class S>
__device__ __forceinline__ void smem_half(S *sk, int lj)
{
    const int j = 1 << lj;
#pragma unroll 4
    for (int c = threadIdx.x; c < P / 2; c += NT) {
        const int lo = ((c >> lj) << (lj + 1)) + (c & (j - 1));
        smem_cx(sk, lo, lo + j);
    }
}

// Sorts NT*E elements held by the CTA (blocked layout); sk holds at least
// pad32(NT*E) elements.
template <int NT, int E, class S>
__device__ __forceinline__ void cta_bitonic_sort(S (&k)[E], S *sk)
{
    constexpr int P = NT * E;
    const int lane = threadIdx.x & 31;
    warp_bitonic_sort<E, S>(k);
    for (int sz = 64 * E, lg = __ffs(64 * E) - 1; sz <= P; sz <<= 1, ++lg) {  // lg = log2(sz)
        regs_to_smem<E, S>(k, sk);
        __syncthreads();
        smem_flip<NT, P, S>(sk, lg - 1);
        __syncthreads();
        for (int lj = lg - 2; (1 << lj) >= 32 * E; --lj) {
            smem_half<NT, P, S>(sk, lj);
            __syncthreads();
        }
        smem_to_regs<E, S>(k, sk);
        __syncthreads();
        for (int j = 16 * E; j >= E; j >>= 1) shfl_half<E, S>(k, j / E, (lane & (j / E)) != 0);
        reg_half<E, E / 2>(k);
    }
}

}  // namespace qs

namespace qs {

// ---------------------------------------------------------------------------
// Register-blocked Bitonic sort with layout transposes.
//
// A group of NG threads (a power of two, >= 32) holds P = NG*E elements, E =
// 2^LE per thread.  A "layout c" keeps the element index bits [c, c+LE) in the
// register index and the other bits, in order, in the thread index:
//   index(g, r) = (g mod 2^c) | r << c | (g >> c) << (c + LE).
// Every compare-exchange then runs between two registers of one thread; to
// reach a stage on index bit d the group moves to a layout containing d by a
// transpose through shared memory (one store and one load per element).
// This is the direction-alternating form of Batcher's network (merge block
// 2^m, stages on bits m-1 .. 0, descending where index bit m is set), which
// needs single-bit stages only.  Padding with the largest key still ends up
// at the tail: it is the largest value, and pads that tie with real keys are
// bit-identical words.
// ---------------------------------------------------------------------------
// Shared-memory slot of element i: one pad word per 128 bytes keeps every
// layout's accesses free of bank conflicts (PSH = 4 for 8-byte keys, 5 for
// 4-byte keys).
template <class S>
__device__ __forceinline__ int padk(int i)
{
    constexpr int PSH = sizeof(S) == 8 ? 4 : 5;
    return i + (i >> PSH);
}

// In layout c the E slots of a thread are base + r*stride (all layouts used
// have c == 0 or c >= PSH, where the padding is linear in r).
template <int LE, class S>
__device__ __forceinline__ void lay_addr(int g, int c, int &base, int &stride)
{
    constexpr int PSH = sizeof(S) == 8 ? 4 : 5;
    const int low = g & ((1 << c) - 1), high = g >> c;
    base = padk<S>(low | (high << (c + LE)));
    stride = c == 0 ? 1 : (1 << c) + (1 << (c - PSH));
}

template <int E, int LE, class S>
__device__ __forceinline__ void lay_store(const S (&k)[E], S *sm, int g, int c)
{
    int base, stride;
    lay_addr<LE, S>(g, c, base, stride);
    S *p = sm + base;
#pragma unroll
    for (int r = 0; r < E; ++r) p[r * stride] = k[r];
}

template <int E, int LE, class S>
__device__ __forceinline__ void lay_load(S (&k)[E], const S *sm, int g, int c)
{
    int base, stride;
    lay_addr<LE, S>(g, c, base, stride);
    const S *p = sm + base;
#pragma unroll
    for (int r = 0; r < E; ++r) k[r] = p[r * stride];
}

__device__ __forceinline__ void group_sync(int bar, int nthreads)
{
    if (nthreads == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}

// Ordered pair: (min, max) ascending, (max, min) descending.
template <bool DESC, class S>
__device__ __forceinline__ void cx_dir(S &a, S &b)
{
    if constexpr (sizeof(S) == 4) {
        const S lo = min(a, b), hi = max(a, b);
        a = DESC ? hi : lo;
        b = DESC ? lo : hi;
    } else {
        const bool sw = DESC ? (a < b) : (b < a);
        const S x = sw ? b : a;
        b = sw ? a : b;
        a = x;
    }
}

// One stage on register bit RB with the same direction for the whole thread.
template <int E, int RB, bool DESC, class S>
__device__ __forceinline__ void reg_stage_u(S (&k)[E])
{
#pragma unroll
    for (int r = 0; r < E; ++r)
        if (!(r & (1 << RB))) cx_dir<DESC, S>(k[r], k[r | (1 << RB)]);
}

// One stage on register bit RB whose direction is register bit MRB.
template <int E, int RB, int MRB, class S>
__device__ __forceinline__ void reg_stage_p(S (&k)[E])
{
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if (r & (1 << RB)) continue;
        if ((r >> MRB) & 1)
            cx_dir<true, S>(k[r], k[r | (1 << RB)]);
        else
            cx_dir<false, S>(k[r], k[r | (1 << RB)]);
    }
}

template <int E, int RB, class S>
__device__ __forceinline__ void reg_stage_rb(S (&k)[E], int mrb, bool tdesc)
{
    switch (mrb) {
    case -1:
        if (tdesc)
            reg_stage_u<E, RB, true, S>(k);
        else
            reg_stage_u<E, RB, false, S>(k);
        break;
    case 1: if constexpr (RB < 1 && E > 2) reg_stage_p<E, RB, 1, S>(k); break;
    case 2: if constexpr (RB < 2 && E > 4) reg_stage_p<E, RB, 2, S>(k); break;
    case 3: if constexpr (RB < 3 && E > 8) reg_stage_p<E, RB, 3, S>(k); break;
    case 4: if constexpr (RB < 4 && E > 16) reg_stage_p<E, RB, 4, S>(k); break;
    default: break;
    }
}

// A stage on register bit rb; mrb = register bit holding the direction, or -1
// when the direction is the same for the whole thread (tdesc).
template <int E, int LE, class S>
__device__ __forceinline__ void reg_stage(S (&k)[E], int rb, int mrb, bool tdesc)
{
    static_assert(LE >= 1 && LE <= 5, "2..32 registers per thread");
    switch (rb) {
    case 0: reg_stage_rb<E, 0, S>(k, mrb, tdesc); break;
    case 1: if constexpr (LE > 1) reg_stage_rb<E, 1, S>(k, mrb, tdesc); break;
    case 2: if constexpr (LE > 2) reg_stage_rb<E, 2, S>(k, mrb, tdesc); break;
    case 3: if constexpr (LE > 3) reg_stage_rb<E, 3, S>(k, mrb, tdesc); break;
    default: if constexpr (LE > 4) reg_stage_rb<E, 4, S>(k, mrb, tdesc); break;
    }
}

// Sorts the P = NG*E elements of a group.  On entry and exit the group holds
// them in layout 0 (blocked: index = g*E + r); sm has room for pad32(P)
// elements; g = thread index inside the group; L = log2(P).
template <int E, int LE, class S>
__device__ void group_bitonic_sort(S (&k)[E], S *sm, int g, int L, int bar, int nthreads)
{
    // Every layout used has c == 0 or c >= LE, so LE >= PSH keeps lay_addr's
    // padding linear in the register index.
    static_assert(LE >= (sizeof(S) == 8 ? 4 : 5), "too few registers per thread for the padded layouts");
    int cur = 0;
    for (int m = 1; m <= L; ++m) {
        for (int d = m - 1; d >= 0; --d) {
            int c = (d / LE) * LE;
            if (c > L - LE) c = L - LE;
            if (c != cur) {
                group_sync(bar, nthreads);
                lay_store<E, LE, S>(k, sm, g, cur);
                group_sync(bar, nthreads);
                lay_load<E, LE, S>(k, sm, g, c);
                cur = c;
            }
            int mrb = -1;
            bool tdesc = false;  // the last merge (m == L) is ascending everywhere
            if (m < L) {
                if (m >= c && m < c + LE)
                    mrb = m - c;
                else
                    tdesc = ((m < c ? (g >> m) : (g >> (m - LE))) & 1) != 0;
            }
            reg_stage<E, LE, S>(k, d - c, mrb, tdesc);
        }
    }
    if (cur != 0) {
        group_sync(bar, nthreads);
        lay_store<E, LE, S>(k, sm, g, cur);
        group_sync(bar, nthreads);
        lay_load<E, LE, S>(k, sm, g, 0);
    }
}

}  // namespace qs
