// Leaf kernel: every part listed by the partition driver is sorted with the
// Bitonic network (Section III-A) into the caller's array, or -- for a
// finished run of equal keys -- copied back from scratch.  Parts larger than
// SMALL keys take one CTA each (registers + shuffles + shared memory); parts
// of at most SMALL keys take one warp each (registers + shuffles only).  The
// tail of a part is padded with the largest sort-space key (Section III-A-3).
#pragma once

#include <type_traits>

#include "qs_bitonic.cuh"
#include "qs_common.cuh"

namespace qs {

// Sort-space element of the leaf network: the integer image of a key
// (KeyOps::to_s), or for key/value pairs the key in the high 32 bits and the
// value's bits in the low 32 bits, compared as a signed 64-bit integer.
template <class Tr>
struct LeafKey {
    using K = typename Tr::K;
    using V = typename Tr::V;
    using Ops = KeyOps<K>;
    using S = typename std::conditional<Tr::KV, long long, typename Ops::S>::type;
    __device__ __forceinline__ static S load(const K *gk, const V *gv, int i)
    {
        if constexpr (Tr::KV)
            return static_cast<long long>((static_cast<unsigned long long>(static_cast<uint32_t>(gk[i])) << 32) |
                                          static_cast<unsigned long long>(static_cast<uint32_t>(gv[i])));
        else
            return Ops::to_s(gk[i]);
    }
    __device__ __forceinline__ static void store(K *ok, V *ov, int i, S s)
    {
        if constexpr (Tr::KV) {
            ok[i] = static_cast<int32_t>(static_cast<uint32_t>(static_cast<unsigned long long>(s) >> 32));
            ov[i] = static_cast<int32_t>(static_cast<uint32_t>(static_cast<unsigned long long>(s)));
        } else {
            ok[i] = Ops::from_s(s);
        }
    }
    __device__ __forceinline__ static S largest()
    {
        if constexpr (Tr::KV)
            return 0x7fffffffffffffffll;
        else
            return Ops::s_largest();
    }
};

template <class Tr>
struct LeafSmem {
    typename LeafKey<Tr>::S keys[Tr::LEAF + Tr::LEAF / 32];
    Leaf leaf;
    long long idx;
};

// A listed part must lie inside the array and fit the kernel that takes it.
template <class Tr>
__device__ bool leaf_ok(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l, bool small)
{
    const int64_t cap = (l.flags & kLeafFinal) ? (small ? a.small_max : kCopyChunk) : (small ? a.small_max : Tr::LEAF);
    const bool ok = l.off >= 0 && l.len > 0 && l.len <= cap && l.off + l.len <= a.n;
    if (!ok) set_error(a.ctrl, kErrInternalIndex, 3);
    return ok;
}

template <class Tr, int E>
__device__ void cta_leaf(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l, LeafSmem<Tr> &sm)
{
    using LK = LeafKey<Tr>;
    using S = typename LK::S;
    constexpr int P = kThreads * E;
    const int src = (l.flags & kLeafScratch) ? 1 : 0;
    const typename Tr::K *gk = a.keys[src] + l.off;
    const typename Tr::V *gv = a.vals[src] + l.off;
    const int len = l.len;
    // Coalesced load into shared memory, tail padded with the largest key.
    for (int i = threadIdx.x; i < P; i += kThreads) sm.keys[pad32(i)] = i < len ? LK::load(gk, gv, i) : LK::largest();
    __syncthreads();
    S k[E];
    smem_to_regs<E, S>(k, sm.keys);
    __syncthreads();
    cta_bitonic_sort<kThreads, E, S>(k, sm.keys);
    regs_to_smem<E, S>(k, sm.keys);
    __syncthreads();
    typename Tr::K *ok = a.keys[0] + l.off;
    typename Tr::V *ov = a.vals[0] + l.off;
    for (int i = threadIdx.x; i < len; i += kThreads) LK::store(ok, ov, i, sm.keys[pad32(i)]);
    __syncthreads();
}

template <class Tr, int E>
__device__ void warp_leaf(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l)
{
    using LK = LeafKey<Tr>;
    using S = typename LK::S;
    const int lane = threadIdx.x & 31;
    const int src = (l.flags & kLeafScratch) ? 1 : 0;
    const typename Tr::K *gk = a.keys[src] + l.off;
    const typename Tr::V *gv = a.vals[src] + l.off;
    const int len = l.len;
    S k[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        k[r] = i < len ? LK::load(gk, gv, i) : LK::largest();
    }
    warp_bitonic_sort<E, S>(k);
    typename Tr::K *ok = a.keys[0] + l.off;
    typename Tr::V *ov = a.vals[0] + l.off;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        if (i < len) LK::store(ok, ov, i, k[r]);
    }
}

template <class Tr, int MinBlocks>
__global__ void __launch_bounds__(kThreads, MinBlocks) leaf_kernel(Args<typename Tr::K, typename Tr::V> a)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    __shared__ LeafSmem<Tr> sm;
    Ctrl *c = a.ctrl;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) sm.idx = ld_relaxed_s32(&c->status);
    __syncthreads();
    if (sm.idx != 0) return;  // the partition phase failed; leave the data alone
    __syncthreads();
    const long long n_large = static_cast<long long>(ld_relaxed_u64(&c->n_large));
    const long long n_small = static_cast<long long>(ld_relaxed_u64(&c->n_small));
    constexpr int kE16 = Tr::LEAF >= kThreads * 16 ? 16 : Tr::LEAF / kThreads;
    constexpr int kE32 = Tr::LEAF >= kThreads * 32 ? 32 : kE16;
    for (;;) {
        if (tid == 0) {
            sm.idx = static_cast<long long>(atomicAdd(&c->claim_large, 1ull));
            if (sm.idx < n_large) {
                sm.leaf = a.leaves[sm.idx];
                if (!leaf_ok<Tr>(a, sm.leaf, false)) sm.leaf.len = 0;
            }
        }
        __syncthreads();
        const long long idx = sm.idx;
        const Leaf l = sm.leaf;
        __syncthreads();
        if (idx >= n_large) break;
        if (l.len == 0) continue;
        if (l.flags & kLeafFinal) {
            const K *gk = a.keys[1] + l.off;
            const V *gv = a.vals[1] + l.off;
            for (int i = tid; i < l.len; i += kThreads) {
                a.keys[0][l.off + i] = gk[i];
                if constexpr (Tr::KV) a.vals[0][l.off + i] = gv[i];
            }
            continue;
        }
        const int len = l.len;
        if (len <= kThreads * 2) cta_leaf<Tr, 2>(a, l, sm);
        else if (len <= kThreads * 4) cta_leaf<Tr, 4>(a, l, sm);
        else if (len <= kThreads * 8) cta_leaf<Tr, 8>(a, l, sm);
        else if (len <= kThreads * 16 || kE32 == kE16) cta_leaf<Tr, kE16>(a, l, sm);
        else cta_leaf<Tr, kE32>(a, l, sm);
    }
    // Small parts: one warp each.
    for (;;) {
        long long idx = 0;
        if (lane == 0) idx = static_cast<long long>(atomicAdd(&c->claim_small, 1ull));
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= n_small) break;
        const Leaf l = a.leaves[a.leaf_cap - 1 - idx];
        if (!leaf_ok<Tr>(a, l, true)) continue;
        if (l.flags & kLeafFinal) {
            for (int i = lane; i < l.len; i += 32) {
                a.keys[0][l.off + i] = a.keys[1][l.off + i];
                if constexpr (Tr::KV) a.vals[0][l.off + i] = a.vals[1][l.off + i];
            }
            continue;
        }
        const int len = l.len;
        if (len <= 32) warp_leaf<Tr, 1>(a, l);
        else if (len <= 64) warp_leaf<Tr, 2>(a, l);
        else if (len <= 128) warp_leaf<Tr, 4>(a, l);
        else if (len <= 256) warp_leaf<Tr, 8>(a, l);
        else warp_leaf<Tr, (Tr::SMALL >= 512 ? 16 : Tr::SMALL / 32)>(a, l);
    }
}

}  // namespace qs
