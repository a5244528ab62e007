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

// Flip stage across lanes: lane l pairs register r with register E-1-r of
// lane l ^ lm.  `upper` is true on the lane holding the higher indices (keeps
// the maximum).  Registers r and E-1-r are exchanged together, so no
// temporary array of E partner values is needed.
template <int E, class S>
__device__ __forceinline__ void shfl_flip(S (&k)[E], int lm, bool upper)
{
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
        const S o_lo = __shfl_xor_sync(0xffffffffu, k[E - 1 - r], lm);
        const S o_hi = __shfl_xor_sync(0xffffffffu, k[r], lm);
        const bool t0 = upper ? (k[r] < o_lo) : (o_lo < k[r]);
        const bool t1 = upper ? (k[E - 1 - r] < o_hi) : (o_hi < k[E - 1 - r]);
        k[r] = t0 ? o_lo : k[r];
        k[E - 1 - r] = t1 ? o_hi : k[E - 1 - r];
    }
    if constexpr (E == 1) {
        const S o = __shfl_xor_sync(0xffffffffu, k[0], lm);
        const bool t = upper ? (k[0] < o) : (o < k[0]);
        k[0] = t ? o : k[0];
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
// at the tail: the last merge is ascending, the pad is the largest value, and
// pads that tie with real keys are bit-identical words.
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

// One stage on register bit RB, every comparator ascending.
template <int E, int RB, class S>
__device__ __forceinline__ void reg_stage_asc(S (&k)[E])
{
#pragma unroll
    for (int r = 0; r < E; ++r)
        if (!(r & (1 << RB))) cx(k[r], k[r | (1 << RB)]);
}

// The stages d = D, D-1, ..., 0 of merge m that exist (d < m), each in the
// layout that holds bit d: c(d) = LE*floor(d/LE), clamped to L-LE.  `cur` is
// the group's current layout.
template <int E, int LE, int L, int D, class S>
__device__ __forceinline__ void merge_stages(S (&k)[E], S *sm, int g, int m, int &cur, int bar, int nthreads)
{
    if constexpr (D >= 0) {
        constexpr int C = (D / LE) * LE > L - LE ? L - LE : (D / LE) * LE;
        if (D < m) {
            if (cur != C) {
                group_sync(bar, nthreads);
                lay_store<E, LE, S>(k, sm, g, cur);
                group_sync(bar, nthreads);
                lay_load<E, LE, S>(k, sm, g, C);
                cur = C;
            }
            reg_stage_asc<E, D - C, S>(k);
        }
        merge_stages<E, LE, L, D - 1, S>(k, sm, g, m, cur, bar, nthreads);
    }
}

// Sorts the P = 2^L elements of a group of NG = P/E threads.  On entry and
// exit the group holds them in layout 0 (blocked: index = g*E + r); sm has
// room for padk(P) elements; g = thread index inside the group.
//
// Batcher's network merges blocks of 2^m elements for m = 1..L, the merge of
// a block descending where index bit m is set.  Instead of comparators of
// both directions, the elements of a descending block are complemented
// (~x reverses the integer order) for the length of its merge, so every
// comparator is the ascending (min, max) of the paper's network; between
// merges m-1 and m an element flips when its index bits m-1 and m differ.
// Merges 1..LE run inside each thread's registers (the flip form above,
// block direction = index bit LE = thread bit 0).
template <int E, int LE, int L, class S>
__device__ void group_bitonic_sort(S (&k)[E], S *sm, int g, int bar, int nthreads)
{
    // Every layout used has c == 0 or c >= LE, so LE >= PSH keeps lay_addr's
    // padding linear in the register index.
    static_assert(LE >= (sizeof(S) == 8 ? 4 : 5), "too few registers per thread for the padded layouts");
    static_assert((1 << LE) == E && L >= LE + 5, "a group is at least one warp");
    const S ones = ~S(0);
    {
        const S f = (g & 1) ? ones : S(0);
#pragma unroll
        for (int r = 0; r < E; ++r) k[r] ^= f;
        reg_merges<E, 2, S>(k);
    }
    int cur = 0;
    for (int m = LE + 1; m <= L; ++m) {
        const int before = (g >> (m - 1 - LE)) & 1;
        const int during = m < L ? (g >> (m - LE)) & 1 : 0;
        const S f = (before ^ during) ? ones : S(0);
#pragma unroll
        for (int r = 0; r < E; ++r) k[r] ^= f;
        merge_stages<E, LE, L, L - 1, S>(k, sm, g, m, cur, bar, nthreads);
    }
}

}  // namespace qs
