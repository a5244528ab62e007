// Device-side building blocks shared by the kernels: key kinds, the
// order-preserving key map, memory-model helpers, TMA bulk copies.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qs_internal.h"

namespace qs {

// ---------------------------------------------------------------------------
// Key kinds.  Every comparison runs in "sort space" S:
//   int32 keys  -> S = int32 (identity);
//   double keys -> S = uint64, the IEEE bit pattern with the sign bit flipped
//                  for non-negative values and all bits flipped for negative
//                  ones.  For doubles without NaN this map is strictly
//                  increasing (-0.0 and +0.0 are the only pair that compare
//                  equal as doubles but differ here; inputs hold no -0.0), so
//                  integer order equals IEEE '<' order and the sorted bits are
//                  exactly those of an IEEE sort.  Integer compares keep the
//                  work off the FP64 pipe, which is narrow on this GPU.
// ---------------------------------------------------------------------------
template <class K>
struct KeyOps;

// The partition compares raw keys against the pivot: int32 as signed
// integers; doubles through their IEEE bits as 64-bit integers -- signed
// compare when the pivot is non-negative, unsigned compare with the direction
// reversed when it is negative (no NaN, no -0.0 among the keys).  The leaf
// sort uses the sort-space map below instead.
template <>
struct KeyOps<int32_t> {
    using S = int32_t;
    using Raw = int32_t;
    using URaw = uint32_t;
    using Vec = int4;
    static constexpr int VW = 4;  // keys per 16-byte vector
    static constexpr bool kSigned = false;  // no sign-dependent compare needed
    __device__ __forceinline__ static Raw raw(int32_t k) { return k; }
    __device__ __forceinline__ static Raw raw_from_bits(uint64_t b) { return static_cast<int32_t>(static_cast<int64_t>(b)); }
    __device__ __forceinline__ static uint64_t to_bits(int32_t k) { return static_cast<uint64_t>(static_cast<int64_t>(k)); }
    __device__ __forceinline__ static S to_s(int32_t k) { return k; }
    __device__ __forceinline__ static int32_t from_s(S s) { return s; }
    __device__ __forceinline__ static S s_largest() { return 0x7fffffff; }
    __device__ __forceinline__ static S s_from_bits(uint64_t b) { return static_cast<int32_t>(static_cast<int64_t>(b)); }
    __device__ __forceinline__ static uint64_t s_to_bits(S s) { return static_cast<uint64_t>(static_cast<int64_t>(s)); }
    __device__ __forceinline__ static void split(const int4 &v, int32_t (&o)[4])
    {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};

template <>
struct KeyOps<double> {
    using S = unsigned long long;
    using Raw = long long;
    using URaw = unsigned long long;
    using Vec = double2;
    static constexpr int VW = 2;
    static constexpr bool kSigned = true;
    __device__ __forceinline__ static Raw raw(double k) { return __double_as_longlong(k); }
    __device__ __forceinline__ static Raw raw_from_bits(uint64_t b) { return static_cast<long long>(b); }
    __device__ __forceinline__ static uint64_t to_bits(double k) { return static_cast<uint64_t>(__double_as_longlong(k)); }
    __device__ __forceinline__ static S to_s(double k)
    {
        const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(k));
        return u ^ (static_cast<unsigned long long>(static_cast<long long>(u) >> 63) | 0x8000000000000000ull);
    }
    __device__ __forceinline__ static double from_s(S s)
    {
        const unsigned long long m = static_cast<unsigned long long>(static_cast<long long>(~s) >> 63) | 0x8000000000000000ull;
        return __longlong_as_double(static_cast<long long>(s ^ m));
    }
    __device__ __forceinline__ static S s_largest() { return ~0ull; }
    __device__ __forceinline__ static S s_from_bits(uint64_t b) { return b; }
    __device__ __forceinline__ static uint64_t s_to_bits(S s) { return s; }
    __device__ __forceinline__ static void split(const double2 &v, double (&o)[2])
    {
        o[0] = v.x;
        o[1] = v.y;
    }
};

// Does a key (raw) go to the lower side?  LE selects '<=' (the equal-key
// pass), NEG a negative double pivot (unsigned, reversed compare).
template <class Ops, bool LE, bool NEG>
__device__ __forceinline__ bool goes_low(typename Ops::Raw k, typename Ops::Raw p)
{
    using U = typename Ops::URaw;
    if constexpr (NEG) {
        return LE ? static_cast<U>(k) >= static_cast<U>(p) : static_cast<U>(k) > static_cast<U>(p);
    } else {
        return LE ? k <= p : k < p;
    }
}

// Compile-time configuration of one element kind.
//   VPT   16-byte vectors per thread per partition tile
//   T     keys per partition tile
//   LEAF  largest part sorted in one CTA's shared memory (power of two); the
//         leaf kernel takes parts of up to MID = 2 * LEAF keys and splits
//         the larger ones once itself (a CTA-local partition through L2)
//   SMALL largest part sorted by a single warp (power of two)
//   PF    true: the next tile is prefetched into a second shared-memory
//         buffer by a TMA bulk copy; false: a tile is loaded straight into
//         registers with 16-byte loads (one shared-memory buffer, for
//         staging only), for tiles too large to double-buffer
//   DT    threads per CTA of the persistent partition kernel
template <class K_, bool KV_, int VPT_, int LEAF_, int SMALL_, bool PF_ = true, int DT_ = kDThreads>
struct Traits {
    using K = K_;
    using V = int32_t;
    using S = typename KeyOps<K_>::S;
    static constexpr bool KV = KV_;
    static constexpr int VW = KeyOps<K>::VW;
    static constexpr int VPT = VPT_;
    static constexpr int E = VPT_ * KeyOps<K_>::VW;  // keys per thread per tile
    static constexpr int DT = DT_;
    static constexpr int DW = DT_ / 32;
    static constexpr int T = DT_ * E;  // keys per partition tile
    static constexpr int LEAF = LEAF_;
    static constexpr int MID = 2 * LEAF_;
    static constexpr int SMALL = SMALL_;
    static constexpr bool PF = PF_;
    static constexpr int NBUF = PF_ ? 2 : 1;  // shared-memory tile buffers
    static_assert(E <= 32, "per-thread flags are kept in one 32-bit mask");
    static_assert(DT_ % 32 == 0 && DT_ >= 128 && DT_ <= 1024, "whole warps; warp 0, the middle warps and the last warp");
};

// ---------------------------------------------------------------------------
// Memory-model helpers.  State written by other CTAs during the persistent
// kernel is read at gpu scope (L2), never through the non-coherent L1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
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
// Fetch-and-add with release (this thread's earlier writes, and the writes it
// has observed through a CTA barrier, become visible first) and acquire (the
// writes released by earlier adders become visible to this thread).
__device__ __forceinline__ unsigned long long atom_add_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.relaxed.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
// SM cycle counter for the profiling slots.  The asm statement is volatile
// with a memory clobber so the compiler keeps it between the barriers and
// memory operations it is meant to bracket.
__device__ __forceinline__ long long prof_clock()
{
    long long t;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(t)::"memory");
    return t;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// mbarrier + 1-D TMA bulk copy (global -> shared).  Used to prefetch the next
// partition tile while the current one is processed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Copies `bytes` (multiple of 16) from 16-byte aligned global memory into
// 16-byte aligned shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Error codes mirrored from qs.h.
constexpr int kErrTimeout = -5;
constexpr int kErrCapacity = -6;
constexpr int kErrDepth = -7;
constexpr int kErrInternalIndex = -7;

__device__ __forceinline__ void set_error(Ctrl *c, int code, int info)
{
    if (atomicCAS(&c->status, 0, code) == 0) c->info = info;
}

// Least time a CTA waits, before it exits, for a bulk copy it issued into
// its own shared memory (whatever QS_OPT_WAIT_LIMIT_NS says).
constexpr uint64_t kDrainFloorNs = 500000000ull;

// Bounded wait on an mbarrier phase by one thread.  Returns false if the
// limit ran out (the error is recorded); the decision is this thread's own,
// so callers inside a barrier sequence make it CTA-uniform before acting.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity, Ctrl *c, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63 && global_ns() - t0 > limit_ns) {
            set_error(c, kErrTimeout, 4);
            return false;
        }
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// Pivot selection.  The paper's experiments use a median of three values
// (Section IV-A); here the median of 64 keys sampled at jittered strides over
// the range: element 32 of the 64 in sorted order.  It is found by rank, not
// by sorting: every lane counts, for its two samples, the samples below and
// not above them, reading all 64 with independent shuffles -- a sort would be
// a chain of ~20 dependent shuffle stages, each queued behind the other
// CTAs' shared-memory traffic.  Called by a full warp (the partition driver
// and the leaf kernel's mid-range stage); returns the pivot's
// raw bits (int32 sign-extended, or IEEE bits).
// ---------------------------------------------------------------------------
template <class K>
__device__ uint64_t sample_median(const K *src, int64_t off, int64_t len, uint64_t salt)
{
    using Ops = KeyOps<K>;
    using S = typename Ops::S;
    const int lane = threadIdx.x & 31;
    S s[2];
    const int64_t stride = len / 64;  // len > 64 for every partition task
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = lane * 2 + r;
        const uint64_t h = mix64(salt * 64 + i);
        const int64_t jitter = static_cast<int64_t>(h % static_cast<uint64_t>(stride > 0 ? stride : 1));
        s[r] = Ops::to_s(__ldcg(src + off + (static_cast<int64_t>(i) * len) / 64 + jitter));
    }
    int lt[2] = {0, 0}, le[2] = {0, 0};
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
        const S o0 = __shfl_sync(0xffffffffu, s[0], j);
        const S o1 = __shfl_sync(0xffffffffu, s[1], j);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            lt[r] += (o0 < s[r] ? 1 : 0) + (o1 < s[r] ? 1 : 0);
            le[r] += (o0 <= s[r] ? 1 : 0) + (o1 <= s[r] ? 1 : 0);
        }
    }
    // Element 32 of the sorted samples is a sample x with lt(x) <= 32 < le(x).
    const bool h0 = lt[0] <= 32 && 32 < le[0];
    const bool h1 = lt[1] <= 32 && 32 < le[1];
    const unsigned m0 = __ballot_sync(0xffffffffu, h0);
    const unsigned m1 = __ballot_sync(0xffffffffu, h1);
    const int from = m0 ? __ffs(m0) - 1 : __ffs(m1) - 1;
    const S x = __shfl_sync(0xffffffffu, h0 ? s[0] : s[1], from);
    return Ops::to_bits(Ops::from_s(x));
}

}  // namespace qs
