// Leaf kernel: every part listed by the partition driver is sorted into the
// caller's array, or -- for a finished run of equal keys -- copied back from
// scratch.  Parts larger than SMALL keys take a group of 32*m threads of a
// 1024-thread CTA (one CTA per SM, the part in shared memory): Bitonic runs
// in registers merged by merge path (qs_merge.cuh); several parts share a
// CTA.  Parts of at most SMALL keys take one warp each and the Bitonic
// network alone (registers + shuffles).  The tail of a part is padded with
// the largest sort-space key (Section III-A-3).
//
// Mid-range parts (LEAF < len <= MID = 2 * LEAF keys, more than one CTA's
// shared memory holds) take the whole CTA for one more quicksort step of
// their own: a sampled pivot, one partition pass from the part's buffer into
// the other one (Section III-B's two write cursors, as in the device-wide
// pass), and the two sides are then sorted like listed parts -- while they
// are still in L2, instead of after one more device-wide pass through HBM.
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
    // The keys, in dynamic shared memory (+64 bytes: a mid-range split shifts
    // each chunk it copies in to the chunk's 16-byte phase).
    static constexpr size_t kDynSmem = sizeof(S) * Tr::LEAF + 64;
};

struct LeafGroup {
    Leaf leaf;
    int start;     // first thread of the group
    int nthreads;  // 32 .. kLThreads, a multiple of 32
    int bar;       // named barrier of the group (groups of one warp use __syncwarp)
};

// Named barriers 1..15 are available to groups (barrier 0 is __syncthreads).
constexpr int kLeafBarriers = 15;


// State of the CTA's mid-range split (one at a time).
struct MidState {
    unsigned tot[2][32];  // per warp: lower-side keys | valid keys << 16 (two chunks in flight)
    uint64_t pivot;       // the pivot's raw bits
    int eq;               // pivot-equal keys of the part
};

template <class Tr>
struct LeafSmem {
    LeafGroup grp[kLThreads / 32];
    Leaf carry;
    int has_carry;
    int ngroups;
    long long idx;
    // Sides of this CTA's last mid-range split still to be sorted (the
    // sortable side on top).  A split runs alone in its pass and pushes at
    // most two sides; the packing loop takes pending sides before any other
    // part and splits the next part only once it is alone in a pass, so the
    // stack holds at most the two sides of one split (a side that does not
    // fit is carried, not pushed back).
    static constexpr int kSides = 8;
    Leaf side[kSides];
    int nside;
    MidState mid;
    alignas(8) unsigned long long mbar;  // completion of a split chunk's bulk copy
    uint32_t mbar_par;                   // parity of its next phase
};

// A listed part must lie inside the array and fit the kernel that takes it.
template <class Tr, bool MID>
__device__ bool leaf_ok(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l, bool small)
{
    const int64_t cap =
        (l.flags & kLeafFinal) ? (small ? a.small_max : kCopyChunk) : (small ? a.small_max : (MID ? Tr::MID : Tr::LEAF));
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
    // 16-byte stores from the first 16-byte boundary on (the keys before it
    // and after the last one one by one): fewer, wider writes, which also
    // carry better over the host link when the output is mapped host memory.
    // Key/value parts need both arrays in the same 16-byte phase.
    using K = typename Tr::K;
    using V = typename Tr::V;
    const uintptr_t kph = reinterpret_cast<uintptr_t>(ok) & 15;
    if (!Tr::KV || kph == (reinterpret_cast<uintptr_t>(ov) & 15)) {
        constexpr int VWS = 16 / static_cast<int>(sizeof(K));
        const int head = static_cast<int>((16 - kph) & 15) / static_cast<int>(sizeof(K));
        const int h = head < len ? head : len;
        const int nvec = (len - h) / VWS;
        const int tail0 = h + nvec * VWS;
        for (int q = g; q < nvec; q += nthreads) {
            K kv[VWS];
            V vv[VWS];
#pragma unroll
            for (int j = 0; j < VWS; ++j) LK::store(kv, vv, j, gs[swz<E>(h + q * VWS + j)]);
            if constexpr (VWS == 2) {
                *reinterpret_cast<double2 *>(ok + h + q * VWS) = make_double2(kv[0], kv[1]);
            } else {
                *reinterpret_cast<int4 *>(ok + h + q * VWS) = make_int4(kv[0], kv[1], kv[2], kv[3]);
                if constexpr (Tr::KV) *reinterpret_cast<int4 *>(ov + h + q * VWS) = make_int4(vv[0], vv[1], vv[2], vv[3]);
            }
        }
        if (g < h) LK::store(ok, ov, g, gs[swz<E>(g)]);
        if (tail0 + g < len) LK::store(ok, ov, tail0 + g, gs[swz<E>(tail0 + g)]);
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int i = g + r * nthreads;
            if (i < len) LK::store(ok, ov, i, gs[swz<E>(i)]);
        }
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

// Sort-space image of a key given by its raw bits (int32 sign-extended, or
// IEEE bits), as sample_median returns it.
template <class K>
__device__ __forceinline__ typename KeyOps<K>::S s_of_bits(uint64_t b)
{
    if constexpr (sizeof(K) == 8)
        return KeyOps<K>::to_s(__longlong_as_double(static_cast<long long>(b)));
    else
        return KeyOps<K>::to_s(static_cast<K>(static_cast<int64_t>(b)));
}

// Copies a finished side from the buffer it sits in to the output (the
// calling group: thread g of ng).
template <class Tr>
__device__ void copy_out(const Args<typename Tr::K, typename Tr::V> &a, int64_t off, int len, int buf, int g, int ng)
{
    if (buf == 0 && !a.out_separate) return;  // already in place
    for (int i = g; i < len; i += ng) {
        a.okeys[off + i] = a.keys[buf][off + i];
        if constexpr (Tr::KV) a.ovals[off + i] = a.vals[buf][off + i];
    }
}

// One quicksort step of a mid-range part by the whole CTA (the packing loop
// gives it every thread, alone in its pass; g = threadIdx.x, named barrier
// `bar`).  The pivot is the median of 64 sampled keys.  A chunk of
// kLThreads*E keys at a time is brought into shared memory (the `smem`
// buffer) by a TMA bulk copy of its 16-byte aligned body, placed at the
// chunk's own 16-byte phase so that any alignment works (the few keys
// outside the body are read from global memory directly); the next chunk's
// copy is issued as soon as the current one has been read, so it lands while
// the current one is placed.  Each thread takes keys g, g + kLThreads, ...,
// compares them, and ranks them with warp ballots: within a warp, the
// lower-side keys of a round take consecutive slots; across warps, a scan of
// the per-warp totals.  Keys are written straight to the other buffer: lower
// side forward from the part's start, upper side backward from its end (the
// two write cursors of Section III-B); the sides are sorted next, so the
// order inside them is free.  Equal keys as in the device-wide pass: if
// nothing is below the pivot the pass is repeated with '<=', whose lower side
// holds only pivot-equal keys and is finished; a side of only pivot-equal
// keys is finished too.  Finished sides are copied to the output at once;
// the others are left on sm.side for the packing loop.
template <class Tr>
__device__ __noinline__ void mid_split(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l, LeafSmem<Tr> &sm,
                                       unsigned char *smem, int bar)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    using Ops = KeyOps<K>;
    using S = typename Ops::S;
    constexpr int E = LeafCfg<Tr>::E;  // keys per thread and chunk
    constexpr int ng = kLThreads, nw = kLThreads / 32, chunk = kLThreads * E;
    constexpr int VK = 16 / static_cast<int>(sizeof(K)), VV = 16 / static_cast<int>(sizeof(V));
    constexpr size_t kVOff = ((static_cast<size_t>(chunk) + VK) * sizeof(K) + 15) & ~static_cast<size_t>(15);
    static_assert(kVOff + (Tr::KV ? (static_cast<size_t>(chunk) + VV) * sizeof(V) : 0) <= LeafCfg<Tr>::kDynSmem,
                  "a chunk and its alignment shift fit the leaf kernel's dynamic shared memory");
    const int g = threadIdx.x;
    const int lane = g & 31, gw = g >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    MidState &ms = sm.mid;
    const int src = (l.flags & kLeafScratch) ? 1 : 0, dst = src ^ 1;
    const int len = l.len;
    const K *gk = a.keys[src] + l.off;
    const V *gv = a.vals[src] + l.off;
    K *dk = a.keys[dst] + l.off;
    V *dv = a.vals[dst] + l.off;
    K *sk = reinterpret_cast<K *>(smem);
    V *sv = reinterpret_cast<V *>(smem + kVOff);
    const bool lead = a.profile && g == 0;
    const long long tq = lead ? prof_clock() : 0;
    // Layout of chunk c0 (every thread computes the same): element i of the
    // chunk sits at sk[pk + i]; [hk, bk) is the body the bulk copy brings
    // (empty if an address check fails: then every key is read directly).
    struct Lay {
        int pk, hk, bk, pv, hv, bv;
        uint32_t bytes;
    };
    auto layout = [&](int c0) {
        Lay y;
        const int nv = len - c0 < chunk ? len - c0 : chunk;
        y.pk = static_cast<int>((reinterpret_cast<uintptr_t>(gk + c0) & 15) / sizeof(K));
        y.hk = (VK - y.pk) % VK;
        if (y.hk > nv) y.hk = nv;
        y.bk = y.hk + (nv - y.hk) / VK * VK;
        const uintptr_t ks = reinterpret_cast<uintptr_t>(gk + c0 + y.hk);
        if (((ks | static_cast<uintptr_t>(smem_addr(sk + y.pk + y.hk))) & 15) != 0) y.bk = y.hk;
        y.bytes = static_cast<uint32_t>((y.bk - y.hk) * sizeof(K));
        y.pv = y.hv = y.bv = 0;
        if constexpr (Tr::KV) {
            y.pv = static_cast<int>((reinterpret_cast<uintptr_t>(gv + c0) & 15) / sizeof(V));
            y.hv = (VV - y.pv) % VV;
            if (y.hv > nv) y.hv = nv;
            y.bv = y.hv + (nv - y.hv) / VV * VV;
            const uintptr_t vs = reinterpret_cast<uintptr_t>(gv + c0 + y.hv);
            if (((vs | static_cast<uintptr_t>(smem_addr(sv + y.pv + y.hv))) & 15) != 0) y.bv = y.hv;
            y.bytes += static_cast<uint32_t>((y.bv - y.hv) * sizeof(V));
        }
        return y;
    };
    auto issue = [&](int c0) {  // thread 0: the bulk copies of chunk c0's bodies
        const Lay y = layout(c0);
        if (y.bytes == 0) return;
        mbar_arrive_expect_tx(&sm.mbar, y.bytes);
        if (y.bk > y.hk)
            bulk_g2s(sk + y.pk + y.hk, gk + c0 + y.hk, static_cast<uint32_t>((y.bk - y.hk) * sizeof(K)), &sm.mbar);
        if constexpr (Tr::KV)
            if (y.bv > y.hv)
                bulk_g2s(sv + y.pv + y.hv, gv + c0 + y.hv, static_cast<uint32_t>((y.bv - y.hv) * sizeof(V)), &sm.mbar);
    };
    uint32_t mpar = sm.mbar_par;
    if (g == 0) issue(0);
    if (gw == 0) {  // the pivot sample's loads overlap the first chunk's copy
        const uint64_t pb =
            sample_median<K>(a.keys[src], l.off, len, static_cast<uint64_t>(l.off) * 0x9E3779B97F4A7C15ull + len);
        if (lane == 0) {
            ms.pivot = pb;
            ms.eq = 0;
            atomicAdd(&a.ctrl->mid_parts, 1ull);
        }
    }
    group_sync(bar, ng);
    if (lead) atomicAdd(&a.ctrl->cycles[31], static_cast<unsigned long long>(prof_clock() - tq));
    const S ps = s_of_bits<K>(ms.pivot);
    bool le = false;  // '<' first
    int low = 0, par = 0;
    for (;;) {
        if (g == 0) atomicAdd(&a.ctrl->mid_keys, static_cast<unsigned long long>(len));
        int lo_base = 0, hi_base = 0;
        for (int c0 = 0; c0 < len; c0 += chunk, par ^= 1) {
            long long tc = lead ? prof_clock() : 0;
            const int nv = len - c0 < chunk ? len - c0 : chunk;
            if (le && c0 == 0 && g == 0) issue(0);  // the '<=' pass reads the part again
            const Lay y = layout(c0);
            if (y.bytes) {  // CTA-uniform; a copy that was issued always lands, so a late one is waited out
                if (!mbar_wait_bounded(&sm.mbar, mpar, a.ctrl, a.wait_limit_ns))
                    mbar_wait_bounded(&sm.mbar, mpar, a.ctrl, kDrainFloorNs);
                mpar ^= 1u;
            }
            K k[E];
            V v[Tr::KV ? E : 1];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int i = r * ng + g;
                k[r] = i < nv ? ((i >= y.hk && i < y.bk) ? sk[y.pk + i] : __ldcg(gk + c0 + i)) : K(0);
                if constexpr (Tr::KV) v[r] = i < nv ? ((i >= y.hv && i < y.bv) ? sv[y.pv + i] : __ldcg(gv + c0 + i)) : 0;
            }
            fence_proxy_async_smem();  // these reads, before a later bulk copy overwrites the buffer
            // This warp's lower-side, valid and pivot-equal keys.
            int wl = 0, wv = 0, eq = 0;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const bool ok = r * ng + g < nv;
                const S s = Ops::to_s(k[r]);
                wl += __popc(__ballot_sync(0xffffffffu, ok && (le ? s <= ps : s < ps)));
                eq += ok && s == ps ? 1 : 0;
                const int rem = nv - (r * ng + gw * 32);  // the valid lanes of a round are a prefix
                wv += rem <= 0 ? 0 : (rem >= 32 ? 32 : rem);
            }
            if (!le) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) eq += __shfl_xor_sync(0xffffffffu, eq, o);
                if (lane == 0 && eq) atomicAdd(&ms.eq, eq);
            }
            // Both counts in one word (each sum stays below 2^16 keys).
            if (lane == 0) ms.tot[par][gw] = static_cast<unsigned>(wl) | (static_cast<unsigned>(wv) << 16);
            if (lead) {
                const long long now = prof_clock();
                atomicAdd(&a.ctrl->cycles[32], static_cast<unsigned long long>(now - tc));
                tc = now;
            }
            group_sync(bar, ng);
            // Every thread has read this chunk: bring the next one meanwhile.
            if (g == 0 && c0 + chunk < len) issue(c0 + chunk);
            if (lead) {
                const long long now = prof_clock();
                atomicAdd(&a.ctrl->cycles[33], static_cast<unsigned long long>(now - tc));
                tc = now;
            }
            // Exclusive scan of the per-warp totals (every warp the same).
            const unsigned t = lane < nw ? ms.tot[par][lane] : 0u;
            unsigned incl = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned x = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += x;
            }
            const unsigned all = __shfl_sync(0xffffffffu, incl, 31);
            const unsigned before = __shfl_sync(0xffffffffu, incl - t, gw);
            const int L = static_cast<int>(all & 0xffffu);
            const int lb = static_cast<int>(before & 0xffffu), vb0 = static_cast<int>(before >> 16);
            int lpre = lo_base + lb;         // lower-side slots before this warp
            int hpre = hi_base + (vb0 - lb);  // upper-side slots before it
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const bool ok = r * ng + g < nv;
                const bool lo = ok && (le ? Ops::to_s(k[r]) <= ps : Ops::to_s(k[r]) < ps);
                const unsigned b = __ballot_sync(0xffffffffu, lo);
                const unsigned vb = __ballot_sync(0xffffffffu, ok);
                const int lr = __popc(b & lt_mask);
                if (ok) {
                    const int pos = lo ? lpre + lr : len - 1 - (hpre + __popc(vb & ~b & lt_mask));
                    dk[pos] = k[r];
                    if constexpr (Tr::KV) dv[pos] = v[r];
                }
                lpre += __popc(b);
                hpre += __popc(vb & ~b);
            }
            lo_base += L;
            hi_base += nv - L;
            if (lead) atomicAdd(&a.ctrl->cycles[34], static_cast<unsigned long long>(prof_clock() - tc));
        }
        low = lo_base;
        // Uniform decision: lo_base and ms.eq are the same in every thread.
        if (low == 0 && !le && ms.eq != len) {
            le = true;
            continue;
        }
        break;
    }
    group_sync(bar, ng);  // the part's stores are visible to the whole group
    if (g == 0) sm.mbar_par = mpar;
    // The two sides in buffer dst: [0, low) and [low, len).
    const int eqn = ms.eq;
    bool fin[2];
    const int so[2] = {0, low}, sl[2] = {low, len - low};
    if (!le) {
        fin[0] = false;
        fin[1] = eqn == len - low;  // the upper side holds only pivot-equal keys (also: all keys equal)
    } else {
        fin[0] = true;  // '<=' after a '<' pass that moved nothing: the lower side equals the pivot
        fin[1] = false;
    }
    for (int i = 0; i < 2; ++i)
        if (sl[i] > 0 && (fin[i] || sl[i] == 1)) copy_out<Tr>(a, l.off + so[i], sl[i], dst, g, ng);
    if (g == 0) {
        // The side that needs another split goes below the other.  (The
        // packing loop reads the stack only between passes.)
        const int order[2] = {sl[0] > Tr::LEAF ? 0 : 1, sl[0] > Tr::LEAF ? 1 : 0};
        for (int j = 0; j < 2; ++j) {
            const int i = order[j];
            if (sl[i] <= 1 || fin[i]) continue;
            if (sm.nside >= LeafSmem<Tr>::kSides) {  // never (see LeafSmem::side)
                set_error(a.ctrl, kErrInternalIndex, 7);
                continue;
            }
            Leaf c;
            c.off = l.off + so[i];
            c.len = sl[i];
            c.flags = dst == 1 ? kLeafScratch : 0;
            sm.side[sm.nside++] = c;
        }
    }
}

// MID: the listed parts may exceed LEAF (QS_OPT_LEAF_MAX above it), so the
// kernel carries the mid-range split; without it the kernel has no trace of
// the stage (the split's call would cost registers around it).
template <class Tr, bool MID>
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
    if (tid == 0) {
        sm.has_carry = 0;
        sm.nside = 0;
        if constexpr (MID) {
            mbar_init(&sm.mbar, 1);
            fence_mbar_init();
            sm.mbar_par = 0;
        }
    }
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
                } else if (sm.nside > 0) {
                    l = sm.side[--sm.nside];  // a side of this CTA's last split: still in L2
                } else {
                    const long long idx = static_cast<long long>(atomicAdd(&c->claim_large, 1ull));
                    if (idx >= n_large) break;
                    l = a.leaves[idx];
                    if (!leaf_ok<Tr, MID>(a, l, false)) continue;
                }
                // A finished run is copied and a mid-range part split by the
                // whole CTA; a part to sort takes 32*m threads, E keys each.
                int need = kLThreads;
                if (!(l.flags & kLeafFinal) && (!MID || l.len <= Tr::LEAF)) need = 32 * ((l.len + 32 * E - 1) / (32 * E));
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
            // once this pass's work is done (one CTA per SM: nothing else
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
            } else if (MID && l.len > Tr::LEAF) {
                const int st = sm.grp[gi].start;
                const long long tm0 = (a.profile && tid == st) ? prof_clock() : 0;
                // Alone in its pass: the group is the whole CTA.
                mid_split<Tr>(a, l, sm, leaf_dyn, sm.grp[gi].bar);
                if (a.profile && tid == st) {
                    atomicAdd(&a.ctrl->cycles[29], static_cast<unsigned long long>(prof_clock() - tm0));
                    atomicAdd(&a.ctrl->cycles[30], 1ull);
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
            if (!leaf_ok<Tr, MID>(a, l, true)) continue;
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
