// Kernels of the hybrid Quicksort hot path for sm_103a.
//
//   setup_kernel   -- resets the control block and seeds the work queue with
//                     the root partition (or the root leaf for small n).
//   driver_kernel  -- persistent kernel (Section III-C, Algorithm 3, made
//                     device-side): CTAs pull tiles of partition tasks from a
//                     FIFO, partition each tile (Section III-B) with a
//                     single-pass scan and decoupled look-back, and the CTA
//                     that completes a task picks pivots for its children and
//                     queues them; parts of at most leaf_max keys go to the
//                     leaf list instead.
//   leaf_kernel    -- sorts every listed part with the Bitonic network
//                     (Section III-A) into the caller's array, or copies a
//                     finished run of equal keys back from scratch.
//
// Partition order inside a task (fixed so the result is deterministic): keys
// going to the lower side keep input order; keys going to the upper side are
// written from the end of the range backwards, i.e. in reverse input order.
// This is what one forward pass with a left write cursor and a right write
// cursor produces (the paper's left_w / right_w).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qs_bitonic.cuh"
#include "qs_internal.h"

namespace qs {

// ---------------------------------------------------------------------------
// Key kinds
// ---------------------------------------------------------------------------
template <class K>
struct KeyOps;

template <>
struct KeyOps<int32_t> {
    using Vec = int4;
    static constexpr int VW = 4;  // keys per 16-byte vector
    __device__ static int32_t largest() { return 0x7fffffff; }
    __device__ static int32_t from_bits(uint64_t b) { return static_cast<int32_t>(static_cast<int64_t>(b)); }
    __device__ static uint64_t to_bits(int32_t k) { return static_cast<uint64_t>(static_cast<int64_t>(k)); }
    __device__ static void split(const int4 &v, int32_t (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};

template <>
struct KeyOps<double> {
    using Vec = double2;
    static constexpr int VW = 2;
    __device__ static double largest() { return __longlong_as_double(0x7ff0000000000000ll); }  // +inf
    __device__ static double from_bits(uint64_t b) { return __longlong_as_double(static_cast<long long>(b)); }
    __device__ static uint64_t to_bits(double k) { return static_cast<uint64_t>(__double_as_longlong(k)); }
    __device__ static void split(const double2 &v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }
};

// Compile-time configuration of one element kind.
//   VPT   16-byte vectors per thread per tile
//   T     keys per partition tile
//   LEAF  largest part handed to the Bitonic kernel (power of two)
//   SMALL largest part sorted by a single warp (power of two)
template <class K_, bool KV_, int VPT_, int LEAF_, int SMALL_>
struct Traits {
    using K = K_;
    using V = int32_t;
    static constexpr bool KV = KV_;
    static constexpr int VW = KeyOps<K>::VW;
    static constexpr int VPT = VPT_;
    static constexpr int T = kThreads * VPT * VW;
    static constexpr int LEAF = LEAF_;
    static constexpr int SMALL = SMALL_;
};

// ---------------------------------------------------------------------------
// Memory-model helpers.  All state written by other CTAs during the
// persistent kernel is read at gpu scope (L2), never through L1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_s32(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s32(int32_t *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_relaxed_s64(const long long *p)
{
    long long v;
    asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_error(Ctrl *c, int code, int info)
{
    if (atomicCAS(&c->status, 0, code) == 0) c->info = info;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Error codes mirrored from qs.h (kept numeric to avoid a dependency).
constexpr int kErrTimeout = -5;
constexpr int kErrCapacity = -6;
constexpr int kErrDepth = -7;
constexpr int kErrInternalIndex = -7;

// ---------------------------------------------------------------------------
// Pivot selection (Section IV-A uses a median of three; here the median of 64
// keys sampled at jittered strides over the range, sorted by one warp with the
// Bitonic network).  Called by a full warp; every lane gets the pivot.
// ---------------------------------------------------------------------------
template <class K>
__device__ K sample_median(const K *src, int64_t off, int64_t len, uint64_t salt)
{
    const int lane = threadIdx.x & 31;
    K s[2];
    int32_t dummy[2] = {0, 0};
    const int64_t stride = len / 64;  // len > 64 for every partition task
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = lane * 2 + r;
        const uint64_t h = mix64(salt * 64 + i);
        const int64_t pos = off + (static_cast<int64_t>(i) * len) / 64 + static_cast<int64_t>(h % static_cast<uint64_t>(stride > 0 ? stride : 1));
        s[r] = __ldcg(src + pos);
    }
    warp_bitonic_sort<2, K, int32_t, false>(s, dummy);
    return __shfl_sync(0xffffffffu, s[0], 16);  // element 32 of 64
}

// ---------------------------------------------------------------------------
// Task creation and leaf listing (called by one thread).
// ---------------------------------------------------------------------------
template <class Tr>
__device__ bool create_task(const Args<typename Tr::K, typename Tr::V> &a, int64_t off, int64_t len,
                            int src, uint64_t pivot_bits, int mode, int depth)
{
    Ctrl *c = a.ctrl;
    if (depth > kMaxDepth) {
        set_error(c, kErrDepth, depth);
        return false;
    }
    const unsigned long long id = atomicAdd(&c->n_tasks, 1ull);
    if (id >= static_cast<unsigned long long>(a.task_cap)) {
        set_error(c, kErrCapacity, 1);
        return false;
    }
    const int64_t w0 = off - ((a.key_phase[src] + off) % Tr::VW);
    const int64_t ntiles = (off + len - w0 + Tr::T - 1) / Tr::T;
    const unsigned long long pool = atomicAdd(&c->pool_cursor, static_cast<unsigned long long>(ntiles));
    if (pool + ntiles > static_cast<unsigned long long>(a.pool_cap)) {
        set_error(c, kErrCapacity, 2);
        return false;
    }
    Task *t = a.tasks + id;
    t->off = off;
    t->len = len;
    t->w0 = w0;
    t->pool = static_cast<int64_t>(pool);
    t->pivot = pivot_bits;
    t->ntiles = static_cast<int32_t>(ntiles);
    t->src = src;
    t->mode = mode;
    t->depth = depth;
    t->next_tile = 0;
    t->tiles_done = 0;
    t->eq = 0;
    t->lt_total = 0;
    __threadfence();
    const unsigned long long slot = atomicAdd(&c->q_tail, 1ull);
    st_release_s32(a.queue + slot, static_cast<int>(id) + 1);
    atomicAdd(&c->part_tasks, 1ull);
    atomicAdd(&c->part_keys, static_cast<unsigned long long>(len));
    atomicMax(&c->max_depth, static_cast<unsigned long long>(depth));
    return true;
}

// Reserves `count` leaf entries on the large (front) or small (back) side.
// Returns the first index, or -1 on overflow (error recorded).
template <class Tr>
__device__ int64_t reserve_leaves(const Args<typename Tr::K, typename Tr::V> &a, int64_t count, bool small)
{
    Ctrl *c = a.ctrl;
    const unsigned long long used =
        small ? atomicAdd(&c->n_small, static_cast<unsigned long long>(count))
              : atomicAdd(&c->n_large, static_cast<unsigned long long>(count));
    // Both sides share one array; check the combined fill after reserving.
    const unsigned long long other = small ? ld_relaxed_u64(&c->n_large) : ld_relaxed_u64(&c->n_small);
    if (used + count + other > static_cast<unsigned long long>(a.leaf_cap)) {
        set_error(c, kErrCapacity, 3);
        return -1;
    }
    return small ? a.leaf_cap - 1 - static_cast<int64_t>(used) : static_cast<int64_t>(used);
}

template <class Tr>
__device__ void push_leaf(const Args<typename Tr::K, typename Tr::V> &a, int64_t off, int64_t len, int flags)
{
    const bool small = len <= a.small_max;
    const int64_t i = reserve_leaves<Tr>(a, 1, small);
    if (i < 0) return;
    Leaf l;
    l.off = off;
    l.len = static_cast<int32_t>(len);
    l.flags = flags;
    a.leaves[small ? i : i] = l;
    if (!(flags & kLeafFinal)) {
        atomicAdd(&a.ctrl->leaf_parts, 1ull);
        atomicAdd(&a.ctrl->leaf_keys, static_cast<unsigned long long>(len));
    }
}

// ---------------------------------------------------------------------------
// Shared memory of the persistent kernel.
// ---------------------------------------------------------------------------
struct WorkItem {
    int kind;  // 0 exit, 1 tile
    int task;
    int tile;
    int ntiles;
    int src, mode;
    int64_t off, len, w0, pool;
    uint64_t pivot;
};

template <class Tr>
struct DriverSmem {
    typename Tr::K keys[Tr::T];
    typename Tr::V vals[Tr::KV ? Tr::T : 1];
    int wcount[Tr::VPT * kWarps];
    long long excl;
    int low_total;
    int eq_total;
    int last;
    int abort;
    WorkItem work;
    // finisher
    int nchild;
    int64_t c_off[2], c_len[2];
    int c_kind[2];  // 0 none, 1 final, 2 leaf, 3 partition (sample pivot), 4 partition (inherit pivot, mode <=)
};

// ---------------------------------------------------------------------------
// Work fetch (thread 0): returns a tile of the task at the queue head, or
// exit when no partition task is pending.  Every wait is bounded.
// ---------------------------------------------------------------------------
template <class Tr>
__device__ WorkItem fetch_work(const Args<typename Tr::K, typename Tr::V> &a)
{
    Ctrl *c = a.ctrl;
    WorkItem w;
    w.kind = 0;
    uint64_t t0 = 0;
    unsigned ns = 64;
    for (;;) {
        if (ld_relaxed_s32(&c->status) != 0) return w;
        const unsigned long long h = ld_relaxed_u64(&c->q_head);
        const unsigned long long tail = ld_relaxed_u64(&c->q_tail);
        if (h < tail) {
            const int id1 = ld_acquire_s32(a.queue + h);
            if (id1 < 0 || id1 > a.task_cap) {
                set_error(c, kErrInternalIndex, 2);
                return w;
            }
            if (id1 != 0) {
                Task *t = a.tasks + (id1 - 1);
                const unsigned long long tile = atomicAdd(&t->next_tile, 1ull);
                const int ntiles = __ldcg(&t->ntiles);
                if (tile < static_cast<unsigned long long>(ntiles)) {
                    w.kind = 1;
                    w.task = id1 - 1;
                    w.tile = static_cast<int>(tile);
                    w.ntiles = ntiles;
                    w.src = __ldcg(&t->src);
                    w.mode = __ldcg(&t->mode);
                    w.off = __ldcg(&t->off);
                    w.len = __ldcg(&t->len);
                    w.w0 = __ldcg(&t->w0);
                    w.pool = __ldcg(&t->pool);
                    w.pivot = __ldcg(reinterpret_cast<const unsigned long long *>(&t->pivot));
                    return w;
                }
                atomicCAS(&c->q_head, h, h + 1);
                t0 = 0;
                continue;
            }
        } else if (ld_relaxed_s64(&c->pending) == 0) {
            return w;
        }
        const uint64_t now = global_ns();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > a.wait_limit_ns) {
            set_error(c, kErrTimeout, 1);
            return w;
        }
        __nanosleep(ns);
        ns = ns < 2048 ? ns * 2 : ns;
    }
}

// ---------------------------------------------------------------------------
// Decoupled look-back by warp 0 (Merrill & Garland).  Returns the number of
// lower-side keys in all preceding tiles of the task, or -1 if the wait ran
// out or another CTA reported an error.
// ---------------------------------------------------------------------------
static __device__ long long lookback(unsigned long long *words, int tile, unsigned long long low, const Ctrl *c,
                              uint64_t limit_ns)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed_u64(words, kFlagPrefix | low);
        return 0;
    }
    if (lane == 0) st_relaxed_u64(words + tile, kFlagAggregate | low);
    long long excl = 0;
    int idx = tile - 1;
    uint64_t t0 = 0;
    for (;;) {
        const int j = idx - lane;
        unsigned long long s = j >= 0 ? ld_relaxed_u64(words + j) : kFlagPrefix;
        int spins = 0;
        while (__any_sync(0xffffffffu, (s >> 62) == 0)) {
            if ((s >> 62) == 0) s = ld_relaxed_u64(words + j);
            if (++spins == 64) {
                spins = 0;
                int bad = 0;
                if (lane == 0) {
                    const uint64_t now = global_ns();
                    if (t0 == 0) t0 = now;
                    const bool late = now - t0 > limit_ns;
                    if (late) set_error(const_cast<Ctrl *>(c), kErrTimeout, 2);
                    bad = late || ld_relaxed_s32(&c->status) != 0;
                }
                if (__shfl_sync(0xffffffffu, bad, 0)) return -1;
            }
        }
        const unsigned pmask = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        const int first = pmask ? __ffs(pmask) - 1 : 31;
        long long v = lane <= first ? static_cast<long long>(s & kCountMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pmask) break;
        idx -= 32;
    }
    if (lane == 0) st_relaxed_u64(words + tile, kFlagPrefix | static_cast<unsigned long long>(excl + low));
    return excl;
}

// ---------------------------------------------------------------------------
// One partition tile (Section III-B on a GPU).  Each thread holds VPT 16-byte
// vectors; vector k of thread t covers tile positions k*NT*VW + t*VW + j, so
// the input order is (k, warp, lane, j).  The compare against the pivot is
// turned into warp ballots whose popcounts give every key its rank among the
// tile's lower-side keys; a CTA scan of the (k, warp) counts and the
// look-back give the global position.  Keys are staged in shared memory in
// output order and written back with coalesced stores.
// Returns 1 if this CTA completed the task, 0 if not, -1 on abort.
// ---------------------------------------------------------------------------
template <class Tr>
__device__ int partition_tile(const Args<typename Tr::K, typename Tr::V> &a, const WorkItem &w,
                              DriverSmem<Tr> &sm)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    using Vec = typename KeyOps<K>::Vec;
    constexpr int VW = Tr::VW, VPT = Tr::VPT, T = Tr::T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;

    const K *__restrict__ sk = a.keys[w.src];
    const V *__restrict__ sv = a.vals[w.src];
    K *__restrict__ dk = a.keys[w.src ^ 1];
    V *__restrict__ dv = a.vals[w.src ^ 1];
    const bool vvec = a.val_vec[w.src] != 0;
    const int64_t off = w.off, end = w.off + w.len;
    const int64_t base = w.w0 + static_cast<int64_t>(w.tile) * T;
    const K pivot = KeyOps<K>::from_bits(w.pivot);
    const bool le = w.mode == kModeLessEqual;

    K key[VPT][VW];
    V val[VPT][VW];
    bool low[VPT][VW];
    bool valid[VPT][VW];
    int eq = 0;

#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        const int64_t e = base + static_cast<int64_t>(k) * kThreads * VW + tid * VW;
        if (e >= off && e + VW <= end) {
            const Vec vk = __ldcg(reinterpret_cast<const Vec *>(sk + e));
            KeyOps<K>::split(vk, key[k]);
#pragma unroll
            for (int j = 0; j < VW; ++j) valid[k][j] = true;
            if constexpr (Tr::KV) {
                if (vvec) {
                    const int4 vv = __ldcg(reinterpret_cast<const int4 *>(sv + e));
                    val[k][0] = vv.x;
                    val[k][1] = vv.y;
                    val[k][2] = vv.z;
                    val[k][3] = vv.w;
                } else {
#pragma unroll
                    for (int j = 0; j < VW; ++j) val[k][j] = __ldcg(sv + e + j);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                const int64_t p = e + j;
                valid[k][j] = p >= off && p < end;
                key[k][j] = valid[k][j] ? __ldcg(sk + p) : K(0);
                if constexpr (Tr::KV) val[k][j] = valid[k][j] ? __ldcg(sv + p) : 0;
            }
        }
#pragma unroll
        for (int j = 0; j < VW; ++j) {
            low[k][j] = valid[k][j] && (le ? !(pivot < key[k][j]) : key[k][j] < pivot);
            eq += (valid[k][j] && key[k][j] == pivot) ? 1 : 0;
        }
    }

    // Warp ballots -> rank of each key among the lower-side keys of its (k, warp) chunk.
    int rank[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        int tot = 0, pre = 0;
#pragma unroll
        for (int j = 0; j < VW; ++j) {
            const unsigned b = __ballot_sync(0xffffffffu, low[k][j]);
            tot += __popc(b);
            pre += __popc(b & lt_mask);
        }
        rank[k] = pre;
        if (lane == 0) sm.wcount[k * kWarps + warp] = tot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) eq += __shfl_xor_sync(0xffffffffu, eq, o);
    if (lane == 0) atomicAdd(&sm.eq_total, eq);
    __syncthreads();

    // Warp 0: exclusive scan of the (k, warp) counts, then the look-back.
    if (warp == 0) {
        static_assert(VPT * kWarps <= 32, "one lane per (vector, warp) count");
        const int v = lane < VPT * kWarps ? sm.wcount[lane] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += n;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane < VPT * kWarps) sm.wcount[lane] = incl - v;
        unsigned long long *words = a.pool + w.pool;
        const long long excl = lookback(words, w.tile, static_cast<unsigned long long>(total), a.ctrl, a.wait_limit_ns);
        if (lane == 0) {
            sm.excl = excl;
            sm.low_total = total;
            sm.abort = excl < 0;
            if (excl >= 0 && w.tile == w.ntiles - 1)
                st_relaxed_u64(&a.tasks[w.task].lt_total, static_cast<unsigned long long>(excl + total));
        }
    }
    __syncthreads();
    if (sm.abort) return -1;

    const int L = sm.low_total;
    const long long excl = sm.excl;
    const int64_t vstart = base > off ? base : off;
    const int64_t vend = base + T < end ? base + T : end;
    const int nvalid = static_cast<int>(vend - vstart);

    // Stage in output order: lower-side keys at [0, L), upper-side keys after.
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        int r = sm.wcount[k * kWarps + warp] + rank[k];
        const int64_t e = base + static_cast<int64_t>(k) * kThreads * VW + tid * VW;
#pragma unroll
        for (int j = 0; j < VW; ++j) {
            if (valid[k][j]) {
                const int q = static_cast<int>(e + j - vstart);  // position among valid keys
                const int s = low[k][j] ? r : L + (q - r);
                sm.keys[s] = key[k][j];
                if constexpr (Tr::KV) sm.vals[s] = val[k][j];
            }
            r += low[k][j] ? 1 : 0;
        }
    }
    __syncthreads();

    const int64_t hpre = (vstart - off) - excl;  // upper-side keys in earlier tiles
    bool bad = false;
    for (int s = tid; s < nvalid; s += kThreads) {
        const int64_t d = s < L ? off + excl + s : end - 1 - (hpre + (s - L));
        if (d < off || d >= end) {  // never taken when the scan is consistent
            bad = true;
            continue;
        }
        dk[d] = sm.keys[s];
        if constexpr (Tr::KV) dv[d] = sm.vals[s];
    }
    if (bad) set_error(a.ctrl, kErrInternalIndex, 1);
    __syncthreads();
    if (tid == 0) {
        Task *t = a.tasks + w.task;
        atomicAdd(&t->eq, static_cast<unsigned long long>(sm.eq_total));
        sm.eq_total = 0;
        __threadfence();
        const unsigned long long done = atomicAdd(&t->tiles_done, 1ull);
        sm.last = done == static_cast<unsigned long long>(w.ntiles - 1);
        if (sm.last) __threadfence();
    }
    __syncthreads();
    return sm.last;
}

// ---------------------------------------------------------------------------
// Completing a task (whole CTA): decide the children, pick their pivots,
// queue them or list them as leaves.  Algorithm 3 recurses on both sides;
// a side of at most leaf_max keys is handed to the Bitonic kernel.
// Equal keys (reading of the paper, which is silent on duplicates): with the
// '<' rule nothing moves when the pivot is the smallest key of the range;
// the range is then re-partitioned with '<=', whose lower side holds only
// keys equal to the pivot and is finished.  A side known to hold only keys
// equal to the pivot is finished too.
// ---------------------------------------------------------------------------
template <class Tr>
__device__ void finish_task(const Args<typename Tr::K, typename Tr::V> &a, const WorkItem &w, DriverSmem<Tr> &sm)
{
    using K = typename Tr::K;
    const int tid = threadIdx.x;
    Task *t = a.tasks + w.task;
    const int dst = w.src ^ 1;
    if (tid == 0) {
        const int64_t lt = static_cast<int64_t>(ld_relaxed_u64(&t->lt_total));
        const int64_t eq = static_cast<int64_t>(ld_relaxed_u64(&t->eq));
        const int64_t off = w.off, len = w.len;
        sm.nchild = 0;
        sm.c_kind[0] = sm.c_kind[1] = 0;
        if (a.partition_only) {
            a.ctrl->lt_result = static_cast<unsigned long long>(lt);
        } else if (w.mode == kModeLess) {
            if (lt == 0) {
                sm.c_off[0] = off;
                sm.c_len[0] = len;
                sm.c_kind[0] = (eq == len) ? 1 : 4;
            } else {
                sm.c_off[0] = off;
                sm.c_len[0] = lt;
                sm.c_kind[0] = 3;
                sm.c_off[1] = off + lt;
                sm.c_len[1] = len - lt;
                sm.c_kind[1] = (len - lt == eq) ? 1 : 3;
            }
        } else {  // '<=' pass after a '<' pass that moved nothing: lower side == pivot
            sm.c_off[0] = off;
            sm.c_len[0] = lt;
            sm.c_kind[0] = 1;
            sm.c_off[1] = off + lt;
            sm.c_len[1] = len - lt;
            sm.c_kind[1] = 3;
        }
        for (int i = 0; i < 2; ++i) {
            if (sm.c_kind[i] == 0) continue;
            if (sm.c_len[i] <= 0) {
                sm.c_kind[i] = 0;
                continue;
            }
            if (sm.c_kind[i] == 3 && sm.c_len[i] <= a.leaf_max) sm.c_kind[i] = 2;
            if (sm.c_kind[i] == 4 && sm.c_len[i] <= a.leaf_max) sm.c_kind[i] = 2;
        }
    }
    __syncthreads();
    int nbig = 0;
    for (int i = 0; i < 2; ++i) {
        const int kind = sm.c_kind[i];
        const int64_t coff = sm.c_off[i], clen = sm.c_len[i];
        if (kind == 1) {
            // Finished run of equal keys: copy back only if it sits in scratch.
            if (dst == 1) {
                const bool small = clen <= a.small_max;
                const int64_t chunks = small ? 1 : (clen + kCopyChunk - 1) / kCopyChunk;
                __shared__ long long first;
                if (tid == 0) {
                    first = reserve_leaves<Tr>(a, chunks, small);
                    atomicAdd(&a.ctrl->copy_keys, static_cast<unsigned long long>(clen));
                }
                __syncthreads();
                if (first >= 0) {
                    for (int64_t q = tid; q < chunks; q += kThreads) {
                        Leaf l;
                        l.off = coff + q * kCopyChunk;
                        const int64_t rem = clen - q * kCopyChunk;
                        l.len = static_cast<int32_t>(small ? clen : (rem < kCopyChunk ? rem : kCopyChunk));
                        l.flags = kLeafFinal | kLeafScratch;
                        a.leaves[small ? first : first + q] = l;
                    }
                }
                __syncthreads();
            }
        } else if (kind == 2) {
            if (tid == 0) push_leaf<Tr>(a, coff, clen, dst == 1 ? kLeafScratch : 0);
        } else if (kind == 3 || kind == 4) {
            uint64_t pbits = w.pivot;
            if (kind == 3 && tid < 32) {
                const K p = sample_median<K>(a.keys[dst], coff, clen,
                                             static_cast<uint64_t>(coff) * 0x2545F4914F6CDD1Dull + clen);
                pbits = KeyOps<K>::to_bits(p);
            }
            if (tid == 0) {
                if (create_task<Tr>(a, coff, clen, dst, pbits, kind == 4 ? kModeLessEqual : kModeLess, __ldcg(&t->depth) + 1))
                    ++nbig;
            }
        }
    }
    if (tid == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctrl->pending),
                  static_cast<unsigned long long>(static_cast<long long>(nbig) - 1));
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Persistent partition kernel.
// ---------------------------------------------------------------------------
template <class Tr, int MinBlocks>
__global__ void __launch_bounds__(kThreads, MinBlocks) driver_kernel(Args<typename Tr::K, typename Tr::V> a)
{
    __shared__ DriverSmem<Tr> sm;
    const int tid = threadIdx.x;
    if (tid == 0) sm.eq_total = 0;
    for (;;) {
        if (tid == 0) sm.work = fetch_work<Tr>(a);
        __syncthreads();
        const WorkItem w = sm.work;
        __syncthreads();
        if (w.kind == 0) break;
        const int r = partition_tile<Tr>(a, w, sm);
        if (r < 0) break;
        if (r == 1) finish_task<Tr>(a, w, sm);
    }
    __syncthreads();
    // Clean exit: every task is finished, so no CTA reads the look-back words
    // or queue slots any more; clear this CTA's share for the next call.
    if (ld_relaxed_s32(&a.ctrl->status) == 0) {
        const unsigned long long used = ld_relaxed_u64(&a.ctrl->pool_cursor);
        const unsigned long long nq = ld_relaxed_u64(&a.ctrl->q_tail);
        const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * kThreads;
        for (unsigned long long i = blockIdx.x * kThreads + tid; i < used; i += stride) a.pool[i] = 0;
        for (unsigned long long i = blockIdx.x * kThreads + tid; i < nq; i += stride) a.queue[i] = 0;
        if (tid == 0) atomicAdd(&a.ctrl->exited, 1ull);
    }
}

// ---------------------------------------------------------------------------
// Setup: one CTA.
// ---------------------------------------------------------------------------
template <class Tr>
__global__ void __launch_bounds__(kThreads) setup_kernel(Args<typename Tr::K, typename Tr::V> a)
{
    using K = typename Tr::K;
    Ctrl *c = a.ctrl;
    const int tid = threadIdx.x;
    if (tid == 0) {
        c->q_head = c->q_tail = 0;
        c->n_tasks = c->pool_cursor = 0;
        c->pending = 0;
        c->n_large = c->n_small = 0;
        c->claim_large = c->claim_small = 0;
        c->status = 0;
        c->info = 0;
        c->part_tasks = c->part_keys = c->leaf_parts = c->leaf_keys = c->copy_keys = c->max_depth = 0;
        c->lt_result = 0;
        c->exited = 0;
        __threadfence();
    }
    __syncthreads();
    if (a.partition_only) {
        if (tid == 0 && create_task<Tr>(a, 0, a.n, 0, a.pivot_bits, kModeLess, 0)) c->pending = 1;
    } else if (a.n > a.leaf_max) {
        uint64_t pbits = 0;
        if (tid < 32) pbits = KeyOps<K>::to_bits(sample_median<K>(a.keys[0], 0, a.n, 0x51ED5EEDull));
        if (tid == 0 && create_task<Tr>(a, 0, a.n, 0, pbits, kModeLess, 0)) c->pending = 1;
    } else if (a.n > 1) {
        if (tid == 0) push_leaf<Tr>(a, 0, a.n, 0);
    }
}

// ---------------------------------------------------------------------------
// Leaf kernel: large parts one per CTA, then small parts one per warp.
// ---------------------------------------------------------------------------
template <class Tr, int E>
__device__ void cta_leaf(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l, typename Tr::K *sk,
                         typename Tr::V *sv)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    constexpr int P = kThreads * E;
    const int src = (l.flags & kLeafScratch) ? 1 : 0;
    const K *gk = a.keys[src] + l.off;
    const V *gv = a.vals[src] + l.off;
    K *ok = a.keys[0] + l.off;
    V *ov = a.vals[0] + l.off;
    const int len = l.len;
    // Coalesced load into shared memory, tail padded with the largest key.
    for (int i = threadIdx.x; i < P; i += kThreads) {
        sk[pad32(i)] = i < len ? gk[i] : KeyOps<K>::largest();
        if constexpr (Tr::KV) sv[pad32(i)] = i < len ? gv[i] : 0;
    }
    __syncthreads();
    K k[E];
    V v[E];
    smem_to_regs<kThreads, E, K, V, Tr::KV>(k, v, sk, sv);
    __syncthreads();
    cta_bitonic_sort<kThreads, E, K, V, Tr::KV>(k, v, sk, sv);
    regs_to_smem<kThreads, E, K, V, Tr::KV>(k, v, sk, sv);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += kThreads) {
        ok[i] = sk[pad32(i)];
        if constexpr (Tr::KV) ov[i] = sv[pad32(i)];
    }
    __syncthreads();
}

template <class Tr, int E>
__device__ void warp_leaf(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    const int lane = threadIdx.x & 31;
    const int src = (l.flags & kLeafScratch) ? 1 : 0;
    const K *gk = a.keys[src] + l.off;
    const V *gv = a.vals[src] + l.off;
    K *ok = a.keys[0] + l.off;
    V *ov = a.vals[0] + l.off;
    const int len = l.len;
    K k[E];
    V v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        k[r] = i < len ? gk[i] : KeyOps<K>::largest();
        v[r] = 0;
        if constexpr (Tr::KV) v[r] = i < len ? gv[i] : 0;
    }
    warp_bitonic_sort<E, K, V, Tr::KV>(k, v);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        if (i < len) {
            ok[i] = k[r];
            if constexpr (Tr::KV) ov[i] = v[r];
        }
    }
}

// A listed part must lie inside the array and fit the kernel that takes it.
template <class Tr>
__device__ bool leaf_ok(const Args<typename Tr::K, typename Tr::V> &a, const Leaf &l, bool small)
{
    const int64_t cap = (l.flags & kLeafFinal) ? (small ? a.small_max : kCopyChunk) : (small ? a.small_max : Tr::LEAF);
    const bool ok = l.off >= 0 && l.len > 0 && l.len <= cap && l.off + l.len <= a.n;
    if (!ok) set_error(a.ctrl, kErrInternalIndex, 3);
    return ok;
}

template <class Tr>
struct LeafSmem {
    typename Tr::K keys[Tr::LEAF + Tr::LEAF / 32];
    typename Tr::V vals[Tr::KV ? Tr::LEAF + Tr::LEAF / 32 : 1];
    Leaf leaf;
    long long idx;
};

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
        if (len <= kThreads * 2) cta_leaf<Tr, 2>(a, l, sm.keys, sm.vals);
        else if (len <= kThreads * 4) cta_leaf<Tr, 4>(a, l, sm.keys, sm.vals);
        else if (len <= kThreads * 8) cta_leaf<Tr, 8>(a, l, sm.keys, sm.vals);
        else if (len <= kThreads * 16 || Tr::LEAF <= kThreads * 16) cta_leaf<Tr, (Tr::LEAF >= kThreads * 16 ? 16 : Tr::LEAF / kThreads)>(a, l, sm.keys, sm.vals);
        else cta_leaf<Tr, (Tr::LEAF >= kThreads * 32 ? 32 : Tr::LEAF / kThreads)>(a, l, sm.keys, sm.vals);
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

// ---------------------------------------------------------------------------
// Host-side launcher for one kind.
// ---------------------------------------------------------------------------
template <class Tr, int DriverMin, int LeafMin>
struct Launcher {
    using K = typename Tr::K;
    using V = typename Tr::V;
    static KernelLimits limits()
    {
        KernelLimits l;
        l.leaf_max = Tr::LEAF;
        l.small_max = Tr::SMALL;
        l.tile = Tr::T;
        l.driver_smem = sizeof(DriverSmem<Tr>);
        l.leaf_smem = sizeof(LeafSmem<Tr>);
        return l;
    }
    static int occ(int which, int *bps)
    {
        if (which == 0)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, driver_kernel<Tr, DriverMin>, kThreads, 0);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, leaf_kernel<Tr, LeafMin>, kThreads, 0);
    }
    static int launch(const Args<K, V> &a, LaunchCfg &cfg)
    {
        cudaStream_t s = static_cast<cudaStream_t>(cfg.stream);
        cudaEvent_t *ev = reinterpret_cast<cudaEvent_t *>(cfg.ev);
        if (cfg.profile) cudaEventRecord(ev[0], s);
        setup_kernel<Tr><<<1, kThreads, 0, s>>>(a);
        if (cfg.profile) cudaEventRecord(ev[1], s);
        if (a.partition_only || a.n > a.leaf_max) driver_kernel<Tr, DriverMin><<<cfg.grid_driver, kThreads, 0, s>>>(a);
        if (cfg.profile) cudaEventRecord(ev[2], s);
        if (!a.partition_only) leaf_kernel<Tr, LeafMin><<<cfg.grid_leaf, kThreads, 0, s>>>(a);
        if (cfg.profile) cudaEventRecord(ev[3], s);
        return static_cast<int>(cudaGetLastError());
    }
};

}  // namespace qs
