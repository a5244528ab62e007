// Leaf kernel: every part listed by the partition driver is sorted into the
// caller's array, or -- for a finished run of equal keys -- copied back from
// scratch.  Parts larger than SMALL keys take a group of 32*m threads of a
// 1024-thread CTA (one CTA per SM, the part in shared memory): Bitonic runs
// in registers merged by merge path (qs_merge.cuh); several parts share a
// CTA.  Parts of at most SMALL keys take one warp each and the Bitonic
// network alone (registers + shuffles).  The tail of a part is padded with
// the largest sort-space key (Section III-A-3).
#pragma once

#include <type_traits>

#include "qs_bitonic.cuh"
#include "qs_common.cuh"
#include "qs_merge.cuh"

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

// Keys per thread of a group: 16 for 64-bit sort keys, 32 for 32-bit ones
// (one 128-byte run each), so a CTA of kLThreads threads holds Tr::LEAF keys.
template <class Tr>
struct LeafCfg {
    using S = typename LeafKey<Tr>::S;
    static constexpr int E = sizeof(S) == 8 ? 16 : 32;
    static_assert(kLThreads * E == Tr::LEAF, "a CTA holds exactly one largest leaf");
    static constexpr size_t kDynSmem = sizeof(S) * Tr::LEAF;  // the keys, in dynamic shared memory
};

struct LeafGroup {
    Leaf leaf;
    int start;     // first thread of the group
    int nthreads;  // 32 .. kLThreads, a multiple of 32
    int bar;       // named barrier of the group (groups of one warp use __syncwarp)
};

// Named barriers 1..15 are available to groups (barrier 0 is __syncthreads).
constexpr int kLeafBarriers = 15;

template <class Tr>
struct LeafSmem {
    LeafGroup grp[kLThreads / 32];
    Leaf carry;
    int has_carry;
    int ngroups;
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

// Sorts one leaf with a group of `nthreads` threads starting at thread
// `start`; the group owns the slice of shared memory of its threads' runs.
template <class Tr>
__device__ void group_leaf(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l,
                           typename LeafKey<Tr>::S *keys, int start, int nthreads, int bar)
{
    using LK = LeafKey<Tr>;
    using S = typename LK::S;
    constexpr int E = LeafCfg<Tr>::E;
    S *gs = keys + start * E;
    const int g = threadIdx.x - start;
    const int src = (l.flags & kLeafScratch) ? 1 : 0;
    const typename Tr::K *gk = a.keys[src] + l.off;
    const typename Tr::V *gv = a.vals[src] + l.off;
    const int len = l.len;
    long long t0 = (a.profile && g == 0) ? prof_clock() : 0;
    // Coalesced loads across the group, tail padded with the largest key.
    S k[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = g + r * nthreads;
        k[r] = i < len ? LK::load(gk, gv, i) : LK::largest();
    }
    if (a.profile && g == 0) {
        const long long t = prof_clock();
        atomicAdd(&a.ctrl->cycles[20], static_cast<unsigned long long>(t - t0));
        t0 = t;
    }
    group_merge_sort<E, S>(k, gs, g, nthreads, bar);
    if (a.profile && g == 0) {
        const long long t = prof_clock();
        atomicAdd(&a.ctrl->cycles[21], static_cast<unsigned long long>(t - t0));
        atomicAdd(&a.ctrl->cycles[22], static_cast<unsigned long long>(nthreads * E - len));  // padding slots
        t0 = t;
    }
    group_sync(bar, nthreads);
    typename Tr::K *ok = a.okeys + l.off;
    typename Tr::V *ov = a.ovals + l.off;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = g + r * nthreads;
        if (i < len) LK::store(ok, ov, i, gs[swz<E>(i)]);
    }
    if (a.profile && g == 0) atomicAdd(&a.ctrl->cycles[23], static_cast<unsigned long long>(prof_clock() - t0));
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
    typename Tr::K *ok = a.okeys + l.off;
    typename Tr::V *ov = a.ovals + l.off;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        if (i < len) LK::store(ok, ov, i, k[r]);
    }
}

template <class Tr>
__global__ void __launch_bounds__(kLThreads, 1) leaf_kernel(Args<typename Tr::K, typename Tr::V> a)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    using S = typename LeafKey<Tr>::S;
    __shared__ LeafSmem<Tr> sm;
    extern __shared__ __align__(128) unsigned char leaf_dyn[];
    S *keys = reinterpret_cast<S *>(leaf_dyn);
    Ctrl *c = a.ctrl;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) sm.idx = ld_relaxed_s32(&c->status);
    __syncthreads();
    if (sm.idx != 0) {
        // The partition phase failed: leave the data alone, but clear the
        // look-back words and ticket owners it used (a failed persistent
        // kernel leaves them set), so that the next call -- possibly issued
        // before the host has seen this error -- starts from a clean state.
        unsigned long long used = ld_relaxed_u64(&c->pool_cursor);
        if (used > static_cast<unsigned long long>(a.pool_cap)) used = static_cast<unsigned long long>(a.pool_cap);
        const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * kLThreads;
        for (unsigned long long i = static_cast<unsigned long long>(blockIdx.x) * kLThreads + tid; i < used; i += stride) {
            a.pool[i] = 0;
            a.owner[i] = 0;
        }
        return;
    }
    __syncthreads();
    const long long n_large = static_cast<long long>(ld_relaxed_u64(&c->n_large));
    const long long n_small = static_cast<long long>(ld_relaxed_u64(&c->n_small));
    constexpr int E = LeafCfg<Tr>::E;
    if (tid == 0) sm.has_carry = 0;
    // Large parts: thread 0 packs parts into thread groups (32 .. kLThreads
    // threads each, a multiple of 32, E keys per thread); a part that does
    // not fit (or finds no named barrier left) is carried over to this CTA's
    // next pass.
    for (;;) {
        const long long tp = (a.profile && tid == 0) ? prof_clock() : 0;
        if (tid == 0) {
            int ng = 0, used = 0, nbar = 0;
            for (;;) {
                Leaf l;
                if (sm.has_carry) {
                    l = sm.carry;
                    sm.has_carry = 0;
                } else {
                    const long long idx = static_cast<long long>(atomicAdd(&c->claim_large, 1ull));
                    if (idx >= n_large) break;
                    l = a.leaves[idx];
                    if (!leaf_ok<Tr>(a, l, false)) continue;
                }
                int need = kLThreads;
                if (!(l.flags & kLeafFinal)) need = 32 * ((l.len + 32 * E - 1) / (32 * E));
                if (used + need > kLThreads || (need > 32 && nbar == kLeafBarriers)) {
                    sm.carry = l;
                    sm.has_carry = 1;
                    break;
                }
                sm.grp[ng].leaf = l;
                sm.grp[ng].start = used;
                sm.grp[ng].nthreads = need;
                sm.grp[ng].bar = need > 32 ? ++nbar : 0;
                ++ng;
                used += need;
                if (used == kLThreads) break;
            }
            sm.ngroups = ng;
            if (a.profile) atomicAdd(&a.ctrl->cycles[19], static_cast<unsigned long long>(prof_clock() - tp));
        }
        __syncthreads();
        const int ng = sm.ngroups;
        if (ng == 0) break;
        if (sm.has_carry) {
            // The part carried over is the next pass's: pull its keys (and
            // values) towards L2 now, so that its loads meet L2 instead of HBM
            // once this pass's sorts are done (one CTA per SM: nothing else
            // hides that latency).
            const Leaf nl = sm.carry;
            const int src = (nl.flags & kLeafScratch) ? 1 : 0;
            const char *kb = reinterpret_cast<const char *>(a.keys[src] + nl.off);
            const int64_t kbytes = static_cast<int64_t>(nl.len) * sizeof(K);
            for (int64_t o = static_cast<int64_t>(tid) * 128; o < kbytes; o += static_cast<int64_t>(kLThreads) * 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(kb + o));
            if constexpr (Tr::KV) {
                const char *vb = reinterpret_cast<const char *>(a.vals[src] + nl.off);
                const int64_t vbytes = static_cast<int64_t>(nl.len) * sizeof(V);
                for (int64_t o = static_cast<int64_t>(tid) * 128; o < vbytes; o += static_cast<int64_t>(kLThreads) * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(vb + o));
            }
        }
        int gi = -1;
        for (int i = 0; i < ng; ++i)
            if (tid >= sm.grp[i].start && tid < sm.grp[i].start + sm.grp[i].nthreads) gi = i;
        if (gi >= 0) {
            const Leaf l = sm.grp[gi].leaf;
            if (l.flags & kLeafFinal) {
                const int src = (l.flags & kLeafScratch) ? 1 : 0;
                const K *gk = a.keys[src] + l.off;
                const V *gv = a.vals[src] + l.off;
                for (int i = tid; i < l.len; i += kLThreads) {
                    a.okeys[l.off + i] = gk[i];
                    if constexpr (Tr::KV) a.ovals[l.off + i] = gv[i];
                }
            } else {
                group_leaf<Tr>(a, l, keys, sm.grp[gi].start, sm.grp[gi].nthreads, sm.grp[gi].bar);
            }
        }
        __syncthreads();
    }
    // Small parts: one warp each, claimed in batches of up to 32 when there
    // are many (one atomic and one coalesced read of the descriptors per
    // batch), one at a time when there are few (so every warp gets work).
    const long long nwarps_all = static_cast<long long>(gridDim.x) * (kLThreads / 32);
    const long long per_warp = n_small / (8 * nwarps_all);
    const int batch = per_warp >= 32 ? 32 : (per_warp < 1 ? 1 : static_cast<int>(per_warp));
    for (;;) {
        long long base = 0;
        if (lane == 0) base = static_cast<long long>(atomicAdd(&c->claim_small, static_cast<unsigned long long>(batch)));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_small) break;
        const int cnt = static_cast<int>(n_small - base < batch ? n_small - base : batch);
        Leaf mine;
        mine.off = 0;
        mine.len = 0;
        mine.flags = 0;
        if (lane < cnt) mine = a.leaves[a.leaf_cap - 1 - (base + lane)];
        for (int q = 0; q < cnt; ++q) {
            Leaf l;
            l.off = __shfl_sync(0xffffffffu, mine.off, q);
            l.len = __shfl_sync(0xffffffffu, mine.len, q);
            l.flags = __shfl_sync(0xffffffffu, mine.flags, q);
            if (!leaf_ok<Tr>(a, l, true)) continue;
            if (l.flags & kLeafFinal) {
                const int src = (l.flags & kLeafScratch) ? 1 : 0;
                for (int i = lane; i < l.len; i += 32) {
                    a.okeys[l.off + i] = a.keys[src][l.off + i];
                    if constexpr (Tr::KV) a.ovals[l.off + i] = a.vals[src][l.off + i];
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
}

}  // namespace qs
