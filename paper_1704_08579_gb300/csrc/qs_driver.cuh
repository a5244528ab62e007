// Persistent partition driver (Section III-C, Algorithm 3, made device-side)
// and its partition tile (Section III-B).
//
// Work model: a partition task is cut into tiles of T keys.  When a task is
// created it reserves a contiguous range of global tickets (its look-back
// words) and publishes, for every ticket, the id of the task.  CTAs claim
// tickets in increasing order with one atomic each; a ticket whose task is
// not published yet is simply waited for.  Every wait therefore points to a
// lower ticket (a tile waits for earlier tiles of its task; a claimed ticket
// waits only for the CTA's current, lower ticket), so waits cannot form a
// cycle.  A CTA claims its next ticket while it still processes the current
// tile and, if that tile is known, prefetches its keys (and values) into
// shared memory with a 1-D TMA bulk copy, so loads overlap the scan, the
// look-back and the stores.
//
// Placement of a tile's keys.  Ordered (qs_partition_*, and sorts with
// QS_OPT_ORDERED): fixed so the result is deterministic -- keys going to the
// lower side keep input order; keys going to the upper side are written from
// the end of the range backwards, i.e. in reverse input order -- what one
// pass with a left write cursor and a right write cursor produces (the
// paper's left_w / right_w); a tile learns how many keys of each side come
// before it from the decoupled look-back.  Unordered (the sort's default): a
// tile claims its lower-side range from the front and its upper-side range
// from the back with one atomic add each on the task's two counters, so
// tiles land in claim order and no tile waits for another; inside a tile the
// order is the ordered one.  Either way the lower side holds exactly the
// keys below the pivot, which is all the recursion needs.
//
// Every written tile is released (its stores ordered by a gpu-scope fence
// before an add on the task's tile counter); the CTA whose release is the
// task's last, in whatever order the tiles finish, completes the task without
// waiting for anyone: it picks the pivots of the children (median of 64
// sampled keys) and queues them, or lists them for the Bitonic kernel when
// they hold at most leaf_max keys.
#pragma once

#include "qs_bitonic.cuh"
#include "qs_common.cuh"

namespace qs {

// ---------------------------------------------------------------------------
// Task creation and leaf listing (called by one thread).
// ---------------------------------------------------------------------------
struct NewTask {
    long long id;
    long long g0;  // first ticket / look-back word
    long long ntiles;
};

// Thread 0: allocates a task and its tickets and writes its fields.  The
// tickets become claimable once publish_task() has run.
template <class Tr>
__device__ bool alloc_task(const Args<typename Tr::K, typename Tr::V> &a, int64_t off, int64_t len, int src,
                           uint64_t pivot_bits, int mode, int depth, NewTask &nt)
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
    const unsigned long long g0 = atomicAdd(&c->pool_cursor, static_cast<unsigned long long>(ntiles));
    if (g0 + ntiles > static_cast<unsigned long long>(a.pool_cap)) {
        set_error(c, kErrCapacity, 2);
        return false;
    }
    Task *t = a.tasks + id;
    t->off = off;
    t->len = len;
    t->w0 = w0;
    t->pool = static_cast<int64_t>(g0);
    t->pivot = pivot_bits;
    t->ntiles = static_cast<int32_t>(ntiles);
    t->src = src;
    t->mode = mode;
    t->depth = depth;
    t->next_tile = 0;
    t->tiles_done = 0;
    t->eq = 0;
    t->lt_total = 0;
    t->hi_total = 0;
    __threadfence();
    atomicAdd(&c->part_tasks, 1ull);
    atomicAdd(&c->part_keys, static_cast<unsigned long long>(len));
    atomicMax(&c->max_depth, static_cast<unsigned long long>(depth));
    nt.id = static_cast<long long>(id);
    nt.g0 = static_cast<long long>(g0);
    nt.ntiles = ntiles;
    return true;
}

// Thread 0: allocates the partition children of a finished task (want[i])
// with one atomic on the task count and one on the ticket cursor and writes
// their fields; the fences of publish_task(), after a CTA barrier, order
// these writes before the tickets become claimable.
template <class Tr>
__device__ void alloc_children(const Args<typename Tr::K, typename Tr::V> &a, const bool (&want)[2],
                               const int64_t (&off)[2], const int64_t (&len)[2], int src, const uint64_t (&pivot)[2],
                               const int (&mode)[2], int depth, NewTask (&nt)[2], int (&ok)[2])
{
    Ctrl *c = a.ctrl;
    ok[0] = ok[1] = 0;
    const int cnt = (want[0] ? 1 : 0) + (want[1] ? 1 : 0);
    if (cnt == 0) return;
    if (depth > kMaxDepth) {
        set_error(c, kErrDepth, depth);
        return;
    }
    int64_t w0[2] = {0, 0}, nti[2] = {0, 0};
    for (int i = 0; i < 2; ++i)
        if (want[i]) {
            w0[i] = off[i] - ((a.key_phase[src] + off[i]) % Tr::VW);
            nti[i] = (off[i] + len[i] - w0[i] + Tr::T - 1) / Tr::T;
        }
    const unsigned long long id = atomicAdd(&c->n_tasks, static_cast<unsigned long long>(cnt));
    const unsigned long long g = atomicAdd(&c->pool_cursor, static_cast<unsigned long long>(nti[0] + nti[1]));
    if (id + cnt > static_cast<unsigned long long>(a.task_cap)) {
        set_error(c, kErrCapacity, 1);
        return;
    }
    if (g + nti[0] + nti[1] > static_cast<unsigned long long>(a.pool_cap)) {
        set_error(c, kErrCapacity, 2);
        return;
    }
    unsigned long long nid = id, ng = g, keys = 0;
    for (int i = 0; i < 2; ++i) {
        if (!want[i]) continue;
        Task *t = a.tasks + nid;
        t->off = off[i];
        t->len = len[i];
        t->w0 = w0[i];
        t->pool = static_cast<int64_t>(ng);
        t->pivot = pivot[i];
        t->ntiles = static_cast<int32_t>(nti[i]);
        t->src = src;
        t->mode = mode[i];
        t->depth = depth;
        t->next_tile = 0;
        t->tiles_done = 0;
        t->eq = 0;
        t->lt_total = 0;
        t->hi_total = 0;
        nt[i].id = static_cast<long long>(nid);
        nt[i].g0 = static_cast<long long>(ng);
        nt[i].ntiles = nti[i];
        ok[i] = 1;
        keys += static_cast<unsigned long long>(len[i]);
        ++nid;
        ng += static_cast<unsigned long long>(nti[i]);
    }
    atomicAdd(&c->part_tasks, static_cast<unsigned long long>(cnt));
    atomicAdd(&c->part_keys, keys);
    atomicMax(&c->max_depth, static_cast<unsigned long long>(depth));
}

// Whole CTA (or one warp: first = lane, stride = 32), after alloc_task() and
// a barrier: makes the task's tickets claimable.
__device__ __forceinline__ void publish_task(const int32_t *owner_c, const NewTask &nt, int first = -1,
                                             int stride = kThreads)
{
    int32_t *owner = const_cast<int32_t *>(owner_c);
    __threadfence();  // order the task's fields (written by thread 0) before its tickets
    for (long long i = first < 0 ? threadIdx.x : first; i < nt.ntiles; i += stride)
        asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(owner + nt.g0 + i), "r"(static_cast<int>(nt.id) + 1)
                     : "memory");
}

// Reserves `count` leaf entries on the large (front) or small (back) side.
// Returns the first index, or -1 on overflow (error recorded).
template <class Tr>
__device__ int64_t reserve_leaves(const Args<typename Tr::K, typename Tr::V> &a, int64_t count, bool small)
{
    Ctrl *c = a.ctrl;
    const unsigned long long used = small ? atomicAdd(&c->n_small, static_cast<unsigned long long>(count))
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
    a.leaves[i] = l;
    if (!(flags & kLeafFinal)) {
        atomicAdd(&a.ctrl->leaf_parts, 1ull);
        atomicAdd(&a.ctrl->leaf_keys, static_cast<unsigned long long>(len));
    }
}

// ---------------------------------------------------------------------------
// Shared memory of the persistent kernel.
// ---------------------------------------------------------------------------
struct WorkItem {
    int kind;  // 0 none/exit, 1 tile
    int task;
    long long ticket;
    int tile;
    int ntiles;
    int src, mode;
    int full;   // tile lies entirely inside the task: TMA bulk load
    int a_pub;  // its look-back aggregate was already published (while it was prefetched)
    int64_t off, len, w0, pool;
    uint64_t pivot;
};


template <class Tr>
struct DriverSmem {
    alignas(128) typename Tr::K kbuf[Tr::NBUF][Tr::T];
    alignas(128) typename Tr::V vbuf[Tr::NBUF][Tr::KV ? Tr::T : 4];
    alignas(8) unsigned long long bar[2];
    int wcount[Tr::VPT * Tr::DW];
    long long excl;
    long long hexcl;  // unordered placement: upper-side keys placed before this tile
    long long first;
    int low_total;
    int eq_total;
    int next_low;  // lower-side count of the prefetched tile (middle warps)
    long long tm[kProfSlots];  // per-phase cycles and counters (profiling on)
    int last;
    int abort;
    WorkItem w[2];  // [0] current, [1] next
    long long next_ticket;  // claimed ticket whose task was not published yet
    NewTask nt[2];
    int nt_ok[2];
    int64_t c_off[2], c_len[2];
    int c_kind[2];  // 0 none, 1 finished (equal keys), 2 leaf, 3 partition (sampled pivot), 4 partition ('<=', same pivot)
    uint64_t pbits[2];  // the children's pivots
    WorkItem wp;    // written tile whose release is deferred
    WorkItem wf;    // task to complete (its last tile was just released)
    int has_prev;   // wp is pending
    int prev_eq;    // pivot-equal keys counted in wp's tile
    int prev_last;  // the release of wp completed its task
};

template <class Tr>
__device__ __forceinline__ void fill_tile(const Args<typename Tr::K, typename Tr::V> &a, WorkItem &w)
{
    const int64_t base = w.w0 + static_cast<int64_t>(w.tile) * Tr::T;
    w.full = base >= w.off && base + Tr::T <= w.off + w.len && (!Tr::KV || a.val_vec[w.src]);
}

// Issues the TMA bulk load of a full tile into buffer `b` (thread 0).
template <class Tr>
__device__ __forceinline__ void issue_tile_load(const Args<typename Tr::K, typename Tr::V> &a, const WorkItem &w,
                                                DriverSmem<Tr> &sm, int b)
{
    if (!Tr::PF || !w.full) return;
    const int64_t base = w.w0 + static_cast<int64_t>(w.tile) * Tr::T;
    constexpr uint32_t kb = Tr::T * sizeof(typename Tr::K);
    constexpr uint32_t vb = Tr::KV ? Tr::T * sizeof(typename Tr::V) : 0;
    fence_proxy_async_smem();  // the buffer was last touched by ordinary loads/stores
    mbar_arrive_expect_tx(&sm.bar[b], kb + vb);
    bulk_g2s(sm.kbuf[b], a.keys[w.src] + base, kb, &sm.bar[b]);
    if constexpr (Tr::KV) bulk_g2s(sm.vbuf[b], a.vals[w.src] + base, vb, &sm.bar[b]);
}

// Thread 0: the tile of ticket g if its task is published (kind 1), else
// kind 0.  `hint` avoids re-reading the fields of the task already in hand.
template <class Tr>
__device__ WorkItem try_resolve(const Args<typename Tr::K, typename Tr::V> &a, long long g, const WorkItem &hint)
{
    WorkItem w = hint;
    w.kind = 0;
    w.ticket = g;
    if (g >= a.pool_cap) return w;  // beyond every ticket that can be published
    if (hint.kind == 1 && g >= hint.pool && g < hint.pool + hint.ntiles) {
        // Another tile of the task in hand: tasks own contiguous ticket
        // ranges, so no need to look the owner up.
        w.tile = static_cast<int>(g - w.pool);
        w.kind = 1;
        w.a_pub = 0;
        fill_tile<Tr>(a, w);
        return w;
    }
    const int id1 = ld_acquire_s32(a.owner + g);
    if (id1 <= 0 || id1 > a.task_cap) {
        if (id1 != 0) set_error(a.ctrl, kErrInternalIndex, 2);
        return w;
    }
    if (!(hint.kind == 1 && hint.task == id1 - 1)) {
        const Task *t = a.tasks + (id1 - 1);
        w.task = id1 - 1;
        w.ntiles = __ldcg(&t->ntiles);
        w.src = __ldcg(&t->src);
        w.mode = __ldcg(&t->mode);
        w.off = __ldcg(&t->off);
        w.len = __ldcg(&t->len);
        w.w0 = __ldcg(&t->w0);
        w.pool = __ldcg(&t->pool);
        w.pivot = __ldcg(reinterpret_cast<const unsigned long long *>(&t->pivot));
    }
    w.tile = static_cast<int>(g - w.pool);
    if (w.tile < 0 || w.tile >= w.ntiles) {
        set_error(a.ctrl, kErrInternalIndex, 6);
        return w;
    }
    w.kind = 1;
    w.a_pub = 0;
    fill_tile<Tr>(a, w);
    return w;
}

// Thread 0: waits (bounded) until ticket g's task is published; kind 0 means
// exit (no partition task is pending any more, or an error was reported).
template <class Tr>
__device__ WorkItem resolve_blocking(const Args<typename Tr::K, typename Tr::V> &a, long long g, const WorkItem &hint)
{
    Ctrl *c = a.ctrl;
    uint64_t t0 = 0;
    unsigned ns = 32;
    if (a.partition_only && g >= __ldcg(&a.tasks[0].ntiles)) {
        // A partition-only call has one task, published before the kernel
        // starts: a ticket past its tiles means there is no work left.
        WorkItem w = hint;
        w.kind = 0;
        return w;
    }
    for (;;) {
        WorkItem w = try_resolve<Tr>(a, g, hint);
        if (w.kind == 1 || ld_relaxed_s32(&c->status) != 0) {
            if (ld_relaxed_s32(&c->status) != 0) w.kind = 0;
            return w;
        }
        // No task left at all: ticket g will never be published.
        if (ld_relaxed_s64(&c->pending) == 0) return w;
        const uint64_t now = global_ns();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > a.wait_limit_ns) {
            set_error(c, kErrTimeout, 1);
            w.kind = 0;
            return w;
        }
        __nanosleep(ns);
        ns = ns < 512 ? ns * 2 : ns;
    }
}

// ---------------------------------------------------------------------------
// Decoupled look-back by warp 0 (Merrill & Garland).  Returns the number of
// lower-side keys in all preceding tiles of the task, or -1 if the wait ran
// out or another CTA reported an error.  Lane l of a window looks at tile
// idx - l; the walk stops at the nearest inclusive prefix behind a run of
// published aggregates.  nwin / nspin count the windows read and the re-reads
// of unpublished words (profiling).
// ---------------------------------------------------------------------------
static __device__ long long lookback(unsigned long long *words, int tile, unsigned long long low, Ctrl *c,
                                     uint64_t limit_ns, bool published, int &nwin, int &nspin)
{
    const int lane = threadIdx.x & 31;
    nwin = nspin = 0;
    if (tile == 0) {
        if (lane == 0 && !published) st_relaxed_u64(words, kFlagPrefix | low);
        return 0;
    }
    if (lane == 0 && !published) st_relaxed_u64(words + tile, kFlagAggregate | low);
    long long excl = 0;
    int idx = tile - 1;
    uint64_t t0 = 0;
    int spins = 0;
    unsigned long long s = idx - lane >= 0 ? ld_relaxed_u64(words + (idx - lane)) : kFlagPrefix;
    for (;;) {
        const unsigned flag = static_cast<unsigned>(s >> 62);
        const unsigned notready = __ballot_sync(0xffffffffu, flag == 0);
        const unsigned pmask = __ballot_sync(0xffffffffu, flag == 2);
        const int first_nr = notready ? __ffs(notready) - 1 : 32;
        const int first_p = pmask ? __ffs(pmask) - 1 : 32;
        if (first_p < first_nr || first_nr == 32) {
            // Lanes 0..last form a ready run: add their counts.
            const int last = first_p < first_nr ? first_p : 31;
            long long v = lane <= last ? static_cast<long long>(s & kCountMask) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            excl += v;
            ++nwin;
            if (first_p < first_nr) break;  // reached an inclusive prefix
            idx -= 32;
            const int j = idx - lane;
            s = j >= 0 ? ld_relaxed_u64(words + j) : kFlagPrefix;
            continue;
        }
        // A tile before the nearest prefix has not published yet: re-read it.
        if (flag == 0) s = ld_relaxed_u64(words + (idx - lane));
        ++nspin;
        if (++spins == 64) {
            spins = 0;
            int bad = 0;
            if (lane == 0) {
                const uint64_t now = global_ns();
                if (t0 == 0) t0 = now;
                const bool late = now - t0 > limit_ns;
                if (late) set_error(c, kErrTimeout, 2);
                bad = late || ld_relaxed_s32(&c->status) != 0;
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) return -1;
        }
    }
    if (lane == 0) st_relaxed_u64(words + tile, kFlagPrefix | static_cast<unsigned long long>(excl + low));
    return excl;
}

// ---------------------------------------------------------------------------
// Compare helpers, instantiated for '<' / '<=' and for the sign of a double
// pivot so that the per-key work is one integer compare.
// ---------------------------------------------------------------------------
template <class Tr, bool LE, bool NEG>
__device__ __forceinline__ uint32_t low_mask(const typename Tr::K (&key)[Tr::E], typename KeyOps<typename Tr::K>::Raw p,
                                             uint32_t validm, int &eq)
{
    using Ops = KeyOps<typename Tr::K>;
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < Tr::E; ++i) {
        const typename Ops::Raw k = Ops::raw(key[i]);
        m |= goes_low<Ops, LE, NEG>(k, p) ? (1u << i) : 0u;
        eq += ((validm >> i) & 1u) && k == p ? 1 : 0;
    }
    return m & validm;
}

// Lower-side count of a prefetched tile in shared memory, by the middle warps
// (1 .. DW-2) during the look-back.
template <class Tr, bool LE, bool NEG>
__device__ __forceinline__ int count_low(const typename Tr::K *buf, typename KeyOps<typename Tr::K>::Raw p)
{
    using Ops = KeyOps<typename Tr::K>;
    using Vec = typename Ops::Vec;
    constexpr int NV = Tr::T / Tr::VW;
    const Vec *v = reinterpret_cast<const Vec *>(buf);
    int cnt = 0;
    for (int i = threadIdx.x - 32; i < NV; i += Tr::DT - 64) {
        typename Tr::K tmp[Tr::VW];
        Ops::split(v[i], tmp);
#pragma unroll
        for (int j = 0; j < Tr::VW; ++j) cnt += goes_low<Ops, LE, NEG>(Ops::raw(tmp[j]), p) ? 1 : 0;
    }
    return cnt;
}

template <class Tr>
__device__ __forceinline__ uint32_t low_mask_any(const typename Tr::K (&key)[Tr::E], uint64_t pivot_bits, int mode,
                                                 uint32_t validm, int &eq)
{
    using Ops = KeyOps<typename Tr::K>;
    const typename Ops::Raw p = Ops::raw_from_bits(pivot_bits);
    const bool le = mode == kModeLessEqual;
    if constexpr (Ops::kSigned) {
        if (p < 0) return le ? low_mask<Tr, true, true>(key, p, validm, eq) : low_mask<Tr, false, true>(key, p, validm, eq);
    }
    return le ? low_mask<Tr, true, false>(key, p, validm, eq) : low_mask<Tr, false, false>(key, p, validm, eq);
}

template <class Tr>
__device__ __forceinline__ int count_low_any(const typename Tr::K *buf, uint64_t pivot_bits, int mode)
{
    using Ops = KeyOps<typename Tr::K>;
    const typename Ops::Raw p = Ops::raw_from_bits(pivot_bits);
    const bool le = mode == kModeLessEqual;
    if constexpr (Ops::kSigned) {
        if (p < 0) return le ? count_low<Tr, true, true>(buf, p) : count_low<Tr, false, true>(buf, p);
    }
    return le ? count_low<Tr, true, false>(buf, p) : count_low<Tr, false, false>(buf, p);
}

// ---------------------------------------------------------------------------
// Release of a written tile (one thread, after a CTA barrier that follows the
// tile's stores): its pivot-equal count, then a gpu-scope fence and an add on
// the task's tile counter (releasing the stores); the last adder fences again
// to acquire everyone's.
// The tile that arrives last completes the task, so no CTA ever waits for
// the others.  The release is deferred into the next tile (see
// partition_tile), where the stores have had time to drain.
// ---------------------------------------------------------------------------
template <class Tr>
__device__ __forceinline__ void release_prev(const Args<typename Tr::K, typename Tr::V> &a, DriverSmem<Tr> &sm)
{
    int last = 0;
    if (sm.has_prev) {
        Task *t = a.tasks + sm.wp.task;
        if (sm.prev_eq) atomicAdd(&t->eq, static_cast<unsigned long long>(sm.prev_eq));
        // The fence releases the tile's stores (and its counts); the last
        // adder's second fence acquires every other tile's.
        const long long t0 = a.profile ? prof_clock() : 0;
        fence_acq_rel_gpu();
        const long long t1 = a.profile ? prof_clock() : 0;
        const unsigned long long done = atom_add_relaxed_u64(&t->tiles_done, 1ull);
        last = done == static_cast<unsigned long long>(sm.wp.ntiles - 1) ? 1 : 0;
        if (a.profile && !a.ordered) {
            const long long t2 = prof_clock();
            sm.tm[9] += t1 - t0;
            sm.tm[10] += t2 - t1;
        }
        if (last) {
            fence_acq_rel_gpu();
            sm.wf = sm.wp;
        }
        sm.has_prev = 0;
    }
    sm.prev_last = last;
}

// ---------------------------------------------------------------------------
// One partition tile.  Vector k of thread t covers tile positions
// k*NT*VW + t*VW + j, so the input order is (k, warp, lane, j).  The pivot
// compare (the paper's vector compare into a mask) becomes warp ballots whose
// popcounts give every key its rank among the tile's lower-side keys; a CTA
// scan of the (k, warp) counts plus the look-back (ordered placement) or the
// tile's two range claims (unordered) give its global position.
// Keys are staged in shared memory in output order and written with
// coalesced stores.  Returns 0; -1 when the wait for the tile's bulk copy
// ran out (that copy may still be in flight); -2 on any other abort.  On
// return sm.prev_last says
// whether the deferred release of the previous tile completed its task
// (sm.wf), which the caller then completes.
// ---------------------------------------------------------------------------
template <class Tr>
__device__ int partition_tile(const Args<typename Tr::K, typename Tr::V> &a, const WorkItem &w, WorkItem &nx,
                              DriverSmem<Tr> &sm, int b, uint32_t &phases)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    using Ops = KeyOps<K>;
    using Vec = typename Ops::Vec;
    constexpr int VW = Tr::VW, VPT = Tr::VPT, T = Tr::T, E = Tr::E;
    constexpr int NC = VPT * Tr::DW;       // (vector, warp) chunk counts
    constexpr int CPL = (NC + 31) / 32;    // chunk counts per lane in the scan
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;

    const int64_t off = w.off, end = w.off + w.len;
    const int64_t base = w.w0 + static_cast<int64_t>(w.tile) * T;

    long long tprev = (a.profile && tid == 0) ? prof_clock() : 0;
#define QS_TICK(slot)                         \
    if (a.profile && tid == 0) {              \
        const long long tnow_ = prof_clock();    \
        sm.tm[slot] += tnow_ - tprev;         \
        tprev = tnow_;                        \
    }

    // Unordered placement: the last warp releases the previous tile first;
    // its fence waits for this SM's earlier stores to drain while the other
    // warps compare.  (Ordered placement releases in the look-back phase,
    // where the middle warps count the next tile meanwhile.)
    if (!a.ordered && warp == Tr::DW - 1) {
        if (lane == 0) {
            const long long trl = a.profile ? prof_clock() : 0;
            release_prev<Tr>(a, sm);
            if (a.profile) sm.tm[5] += prof_clock() - trl;
        }
        __syncwarp();
    }

    K key[E];
    V val[Tr::KV ? E : 1];
    uint32_t validm = 0;
    // A timed-out wait is a per-thread event.  The thread that saw it keeps
    // going with no keys (every warp still takes part in every ballot and
    // barrier below), and the whole CTA abandons the tile at the barrier
    // after the ballots (__syncthreads_or), so no thread leaves a barrier
    // sequence the others are in.  The phase bit is flipped only once the
    // whole CTA has consumed the phase; on abort it stays, so the exit drain
    // waits for the very copy that was late.
    bool landed = true;
    if (!Tr::PF && w.full) {
        // Register tile: 16-byte loads straight from global memory, coalesced
        // across the CTA (the tile's start is 16-byte aligned, see fill_tile).
        const Vec *gk = reinterpret_cast<const Vec *>(a.keys[w.src] + base);
        const int4 *gv = reinterpret_cast<const int4 *>(a.vals[w.src] + base);
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            K tmp[VW];
            Ops::split(__ldcg(gk + k * Tr::DT + tid), tmp);
#pragma unroll
            for (int j = 0; j < VW; ++j) key[k * VW + j] = tmp[j];
            if constexpr (Tr::KV) {
                const int4 vv = __ldcg(gv + k * Tr::DT + tid);
                val[k * VW + 0] = vv.x;
                val[k * VW + 1] = vv.y;
                val[k * VW + 2] = vv.z;
                val[k * VW + 3] = vv.w;
            }
        }
        validm = E == 32 ? 0xffffffffu : ((1u << E) - 1u);
        QS_TICK(1);
    } else if (w.full) {
        landed = mbar_wait_bounded(&sm.bar[b], (phases >> b) & 1u, a.ctrl, a.wait_limit_ns);
        QS_TICK(1);
        const Vec *sv = reinterpret_cast<const Vec *>(sm.kbuf[b]);
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            K tmp[VW];
            if (landed) {
                Ops::split(sv[k * Tr::DT + tid], tmp);
            } else {
#pragma unroll
                for (int j = 0; j < VW; ++j) tmp[j] = K(0);
            }
#pragma unroll
            for (int j = 0; j < VW; ++j) key[k * VW + j] = tmp[j];
            if constexpr (Tr::KV) {
                const int4 vv = landed ? reinterpret_cast<const int4 *>(sm.vbuf[b])[k * Tr::DT + tid]
                                       : make_int4(0, 0, 0, 0);
                val[k * VW + 0] = vv.x;
                val[k * VW + 1] = vv.y;
                val[k * VW + 2] = vv.z;
                val[k * VW + 3] = vv.w;
            }
        }
        validm = landed ? (E == 32 ? 0xffffffffu : ((1u << E) - 1u)) : 0u;
    } else {
        const K *__restrict__ sk = a.keys[w.src];
        const V *__restrict__ svv = a.vals[w.src];
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int64_t e = base + static_cast<int64_t>(k) * Tr::DT * VW + tid * VW;
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                const int64_t p = e + j;
                const bool ok = p >= off && p < end;
                key[k * VW + j] = ok ? __ldcg(sk + p) : K(0);
                if constexpr (Tr::KV) val[k * VW + j] = ok ? __ldcg(svv + p) : 0;
                validm |= ok ? (1u << (k * VW + j)) : 0u;
            }
        }
    }
    int eq = 0;
    const uint32_t lowm = low_mask_any<Tr>(key, w.pivot, w.mode, validm, eq);

    // Warp ballots -> rank of each key among the lower-side keys of its (k, warp) chunk.
    int rank[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        int tot = 0, pre = 0;
#pragma unroll
        for (int j = 0; j < VW; ++j) {
            const unsigned bb = __ballot_sync(0xffffffffu, (lowm >> (k * VW + j)) & 1u);
            tot += __popc(bb);
            pre += __popc(bb & lt_mask);
        }
        rank[k] = pre;
        if (lane == 0) sm.wcount[k * Tr::DW + warp] = tot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) eq += __shfl_xor_sync(0xffffffffu, eq, o);
    if (lane == 0 && eq) atomicAdd(&sm.eq_total, eq);
    if (a.profile && tid == 0) sm.tm[18] += prof_clock() - tprev;  // own work, before the barrier
    if (__syncthreads_or(landed ? 0 : 1)) return -1;  // CTA-uniform: some thread's wait ran out
    if (Tr::PF && w.full) phases ^= 1u << b;
    if constexpr (!Tr::PF) {
        // Register tile: the next tile (resolved by thread 0 before this
        // one, visible since the barrier) is pulled towards L2 now, a whole
        // placement + write-out phase before its loads are issued.
        if (nx.kind == 1 && nx.full) {
            const int64_t nbase = nx.w0 + static_cast<int64_t>(nx.tile) * T;
            const char *kb = reinterpret_cast<const char *>(a.keys[nx.src] + nbase);
            constexpr int kLines = T * static_cast<int>(sizeof(K)) / 128;
#pragma unroll
            for (int q = tid; q < kLines; q += Tr::DT) asm volatile("prefetch.global.L2 [%0];" ::"l"(kb + q * 128));
            if constexpr (Tr::KV) {
                const char *vb = reinterpret_cast<const char *>(a.vals[nx.src] + nbase);
                constexpr int vLines = T * static_cast<int>(sizeof(V)) / 128;
#pragma unroll
                for (int q = tid; q < vLines; q += Tr::DT)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(vb + q * 128));
            }
        }
    }
    QS_TICK(2);
    const long long tph = a.profile ? prof_clock() : 0;  // start of the placement phase

    // Staging in output order (lower-side keys at [0, L), upper-side keys
    // after them) depends only on this tile's own counts, not on the global
    // offset; so warp 0 scans the chunk counts and releases the other warps
    // (named barrier 2) before it starts the look-back or the range claims,
    // and they stage their keys meanwhile.
    const int64_t vstart = base > off ? base : off;
    const int64_t vend = base + T < end ? base + T : end;
    const int nvalid = static_cast<int>(vend - vstart);
    const int vofs = static_cast<int>(vstart - base);  // window slots before the first valid key
    K *stage_k = sm.kbuf[Tr::PF ? b : 0];
    V *stage_v = sm.vbuf[Tr::PF ? b : 0];
    auto stage = [&](int L) {
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            int r = sm.wcount[k * Tr::DW + warp] + rank[k];
            const int e = k * Tr::DT * VW + tid * VW - vofs;
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                const int i = k * VW + j;
                const bool lo = (lowm >> i) & 1u;
                if ((validm >> i) & 1u) {
                    const int s = lo ? r : L + (e + j - r);
                    stage_k[s] = key[i];
                    if constexpr (Tr::KV) stage_v[s] = val[i];
                }
                r += lo ? 1 : 0;
            }
        }
    };
    if (warp == 0) {
        int v[CPL];
        int sum = 0;
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int idx = lane * CPL + i;
            v[i] = idx < NC ? sm.wcount[idx] : 0;
            sum += v[i];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += n;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int run = incl - sum;
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int idx = lane * CPL + i;
            if (idx < NC) sm.wcount[idx] = run;
            run += v[i];
        }
        if (lane == 0) sm.low_total = total;
        __syncwarp();
        asm volatile("bar.arrive 2, %0;" ::"n"(Tr::DT) : "memory");
        const long long tlb = a.profile ? prof_clock() : 0;
        if (a.ordered) {
            int nwin, nspin;
            const long long excl = lookback(a.pool + w.pool, w.tile, static_cast<unsigned long long>(total), a.ctrl,
                                            a.wait_limit_ns, w.a_pub != 0, nwin, nspin);
            if (a.profile && lane == 0) {
                sm.tm[8] += prof_clock() - tlb;
                sm.tm[10] += nwin;
                sm.tm[11] += nspin;
            }
            if (lane == 0) {
                sm.excl = excl;
                sm.abort = excl < 0;
                if (excl >= 0 && w.tile == w.ntiles - 1)
                    st_relaxed_u64(&a.tasks[w.task].lt_total, static_cast<unsigned long long>(excl + total));
                if (excl >= 0 && w.tile == w.ntiles - 1 && a.partition_only)
                    a.ctrl->lt_result = static_cast<unsigned long long>(excl + total);  // the split
            }
            const long long tst = a.profile ? prof_clock() : 0;
            stage(total);
            if (a.profile && lane == 0) {
                const long long now = prof_clock();
                sm.tm[16] += now - tst;
                sm.tm[14] += now - tph;
            }
        } else {
            // Unordered placement: lane 0 claims the tile's lower-side range
            // and lane 1 its upper-side range on the task's two counters; the
            // replies arrive while the warp stages its keys.
            Task *t = a.tasks + w.task;
            const unsigned long long cnt =
                static_cast<unsigned long long>(lane == 0 ? total : nvalid - total);
            unsigned long long got = 0;
            if (lane < 2 && cnt) got = atomicAdd(lane == 0 ? &t->lt_total : &t->hi_total, cnt);
            const long long tst = a.profile ? prof_clock() : 0;
            stage(total);
            const long long excl = static_cast<long long>(__shfl_sync(0xffffffffu, got, 0));
            const long long hexcl = static_cast<long long>(__shfl_sync(0xffffffffu, got, 1));
            if (lane == 0) {
                sm.excl = excl;
                sm.hexcl = hexcl;
                sm.abort = 0;
            }
            if (a.profile && lane == 0) {
                const long long now = prof_clock();
                sm.tm[8] += now - tlb;
                sm.tm[16] += now - tst;
                sm.tm[14] += now - tph;
            }
        }
    } else if (warp < Tr::DW - 1) {
        if (Tr::PF && a.ordered && nx.kind == 1 && nx.full && !nx.a_pub) {
            // The middle warps first count the prefetched next tile and
            // publish its aggregate, so tiles after it never wait for this CTA
            // to finish the current tile.
            const long long tmb = (a.profile && tid == 32) ? prof_clock() : 0;
            const bool landed = mbar_wait_bounded(&sm.bar[b ^ 1], (phases >> (b ^ 1)) & 1u, a.ctrl, a.wait_limit_ns);
            if (a.profile && tid == 32) sm.tm[9] += prof_clock() - tmb;
            if (landed) {
                int cnt = count_low_any<Tr>(sm.kbuf[(b ^ 1) % Tr::NBUF], nx.pivot, nx.mode);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                if (lane == 0) atomicAdd(&sm.next_low, cnt);
            }
            asm volatile("bar.sync 1, %0;" ::"n"(Tr::DT - 64) : "memory");
            if (tid == 32) {
                const unsigned long long c = static_cast<unsigned long long>(sm.next_low);
                st_relaxed_u64(a.pool + nx.pool + nx.tile, (nx.tile == 0 ? kFlagPrefix : kFlagAggregate) | c);
                sm.next_low = 0;
                nx.a_pub = 1;
            }
        }
        asm volatile("bar.sync 2, %0;" ::"n"(Tr::DT) : "memory");  // chunk offsets are ready
        stage(sm.low_total);
        if (a.profile && tid == 32) sm.tm[12] += prof_clock() - tph;
    } else {
        if (a.ordered) {
            if (lane == 0) {
                const long long trl = a.profile ? prof_clock() : 0;
                release_prev<Tr>(a, sm);
                if (a.profile) sm.tm[5] += prof_clock() - trl;
            }
            __syncwarp();
        }
        asm volatile("bar.sync 2, %0;" ::"n"(Tr::DT) : "memory");  // chunk offsets are ready
        const long long tst = a.profile ? prof_clock() : 0;
        stage(sm.low_total);
        if (a.profile && lane == 0) {
            const long long now = prof_clock();
            sm.tm[17] += now - tst;
            sm.tm[15] += now - tph;
        }
    }
    __syncthreads();
    QS_TICK(3);
    if (sm.abort) return -2;  // the tile's keys were consumed; the look-back gave up
    const int L = sm.low_total;
    const long long excl = sm.excl;

    // Lower side: [off + excl, +L); upper side (reverse order) ends at
    // end - 1 - hpre, where hpre = upper-side keys placed before this tile
    // (ordered: those of the earlier tiles).
    // A partition-only call writes its lower side in place, into the buffer
    // it reads: with ordered placement a tile's lower-side keys land at or
    // before the end of its own window, in windows that have been read
    // already (this tile's, and earlier tiles' -- its look-back finished only
    // after every earlier tile published a count, which each tile does only
    // once its keys are loaded).  Only the upper side goes through scratch.
    const int64_t hpre = a.ordered ? (vstart - off) - excl : sm.hexcl;
    const int H = nvalid - L;
    if (excl >= 0 && off + excl + L <= end && hpre >= 0 && hpre + H <= w.len) {
        const int lo_buf = a.partition_only ? w.src : (w.src ^ 1);
        K *__restrict__ lo_k = a.keys[lo_buf] + (off + excl);
        K *__restrict__ hi_k = a.keys[w.src ^ 1] + (end - 1 - hpre + L);  // key s >= L goes to hi_k - s
        V *__restrict__ lo_v = a.vals[lo_buf] + (off + excl);
        V *__restrict__ hi_v = a.vals[w.src ^ 1] + (end - 1 - hpre + L);
        for (int s = tid; s < nvalid; s += Tr::DT) {
            const bool lo = s < L;
            *(lo ? lo_k + s : hi_k - s) = stage_k[s];
            if constexpr (Tr::KV) *(lo ? lo_v + s : hi_v - s) = stage_v[s];
        }
    } else if (tid == 0) {
        set_error(a.ctrl, kErrInternalIndex, 1);  // never taken when the scan is consistent
    }
    __syncthreads();
    QS_TICK(4);
    if (tid == 0) {  // this tile's release is deferred into the next tile
        sm.wp = w;
        sm.prev_eq = sm.eq_total;
        sm.eq_total = 0;
        // A partition-only call completes no task (its split is recorded by
        // its last tile, its CTAs leave when the tickets run out), so its
        // tiles need no release.
        sm.has_prev = a.partition_only ? 0 : 1;
    }
    __syncthreads();
#undef QS_TICK
    if (a.profile && tid == 0) sm.tm[7] += 1;
    return 0;
}

// ---------------------------------------------------------------------------
// Completing a task (whole CTA): decide the children, pick their pivots,
// queue them or list them as leaves.  Algorithm 3 recurses on both sides; a
// side of at most leaf_max keys goes to the Bitonic kernel.
// Equal keys (the paper is silent on duplicates): with the '<' rule nothing
// moves when the pivot is the smallest key of the range; the range is then
// partitioned again with '<=', whose lower side holds only keys equal to the
// pivot and is finished.  A side known to hold only keys equal to the pivot
// (its size equals the count of pivot-equal keys) is finished too.
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
            if ((sm.c_kind[i] == 3 || sm.c_kind[i] == 4) && sm.c_len[i] <= a.leaf_max) sm.c_kind[i] = 2;
        }
    }
    __syncthreads();
    // Children that are partition tasks: their pivots (warp i + 1 samples
    // child i), then thread 0 allocates both, then the whole CTA publishes
    // their tickets.  Warp 0, which holds thread 0 (ticket claims, and the
    // per-phase counters when profiling), stays out of the sampling: with
    // profiling on its samples took 22.8 k cycles against 4.6 k on another
    // warp (unprofiled sorts: the same time within noise).
    long long tf = (a.profile && tid == 0) ? prof_clock() : 0;
    const int wi = (tid >> 5) - 1;
    if (wi >= 0 && wi < 2) {
        uint64_t pb = w.pivot;
        if (sm.c_kind[wi] == 3)
            pb = sample_median<K>(a.keys[dst], sm.c_off[wi], sm.c_len[wi],
                                  static_cast<uint64_t>(sm.c_off[wi]) * 0x2545F4914F6CDD1Dull + sm.c_len[wi]);
        if ((tid & 31) == 0) sm.pbits[wi] = pb;
    }
    __syncthreads();
    if (tid == 0) {
        if (a.profile) {
            const long long now = prof_clock();
            sm.tm[26] += now - tf;
            tf = now;
        }
        bool want[2];
        int64_t coff[2], clen[2];
        uint64_t piv[2];
        int mode[2];
        for (int i = 0; i < 2; ++i) {
            const int kind = sm.c_kind[i];
            want[i] = kind == 3 || kind == 4;
            coff[i] = sm.c_off[i];
            clen[i] = sm.c_len[i];
            piv[i] = sm.pbits[i];
            mode[i] = kind == 4 ? kModeLessEqual : kModeLess;
            if (kind == 2) push_leaf<Tr>(a, sm.c_off[i], sm.c_len[i], dst == 1 ? kLeafScratch : 0);
        }
        alloc_children<Tr>(a, want, coff, clen, dst, piv, mode, __ldcg(&t->depth) + 1, sm.nt, sm.nt_ok);
        sm.low_total = sm.nt_ok[0] + sm.nt_ok[1];
        if (a.profile) {
            const long long now = prof_clock();
            sm.tm[27] += now - tf;
            tf = now;
        }
    }
    __syncthreads();
    for (int i = 0; i < 2; ++i)
        if (sm.nt_ok[i]) publish_task(a.owner, sm.nt[i], -1, Tr::DT);
    if (a.profile && tid == 0) sm.tm[28] += prof_clock() - tf;
    for (int i = 0; i < 2; ++i) {
        // Finished run of equal keys: copy back if it sits in scratch, or
        // wherever it sits when the result goes to a separate array.
        if (sm.c_kind[i] != 1 || (dst != 1 && !a.out_separate)) continue;
        const int64_t coff = sm.c_off[i], clen = sm.c_len[i];
        const bool small = clen <= a.small_max;
        const int64_t chunks = small ? 1 : (clen + kCopyChunk - 1) / kCopyChunk;
        __syncthreads();
        if (tid == 0) {
            sm.first = reserve_leaves<Tr>(a, chunks, small);
            atomicAdd(&a.ctrl->copy_keys, static_cast<unsigned long long>(clen));
        }
        __syncthreads();
        const long long first = sm.first;
        if (first >= 0) {
            for (int64_t q = tid; q < chunks; q += Tr::DT) {
                Leaf l;
                l.off = coff + q * kCopyChunk;
                const int64_t rem = clen - q * kCopyChunk;
                l.len = static_cast<int32_t>(small ? clen : (rem < kCopyChunk ? rem : kCopyChunk));
                l.flags = kLeafFinal | (dst == 1 ? kLeafScratch : 0);
                a.leaves[small ? first : first + q] = l;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        // This task is done; its partition children are pending.
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctrl->pending),
                  static_cast<unsigned long long>(static_cast<long long>(sm.low_total) - 1));
    }
    __syncthreads();
}

// Releases the deferred tile now (whole CTA) and completes its task if it was
// the last one.
template <class Tr>
__device__ void flush_release(const Args<typename Tr::K, typename Tr::V> &a, DriverSmem<Tr> &sm)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long trl = a.profile ? prof_clock() : 0;
        release_prev<Tr>(a, sm);
        if (a.profile) sm.tm[5] += prof_clock() - trl;
    }
    __syncthreads();
    if (sm.prev_last) finish_task<Tr>(a, sm.wf, sm);
}

// ---------------------------------------------------------------------------
// Persistent partition kernel.
// ---------------------------------------------------------------------------
template <class Tr, int MinBlocks>
__global__ void __launch_bounds__(Tr::DT, MinBlocks) driver_kernel(Args<typename Tr::K, typename Tr::V> a)
{
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    DriverSmem<Tr> &sm = *reinterpret_cast<DriverSmem<Tr> *>(dyn_smem);
    const int tid = threadIdx.x;
    uint32_t phases = 0;   // bit b: parity of the next completion of bar[b]
    uint32_t pending = 0;  // bit b: a bulk load into buffer b is issued and not yet consumed
    long long t_wait = a.profile ? prof_clock() : 0;
    // Unordered placement: thread 0 claims each ticket one tile early, so the
    // claim's round trip is hidden behind a whole tile.  (With ordered
    // placement a held ticket would delay the look-back of the tiles after it.)
    long long g_ahead = 0;
    if (tid == 0) {
        for (int i = 0; i < kProfSlots; ++i) sm.tm[i] = 0;
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
        sm.eq_total = 0;
        sm.next_low = 0;
        sm.has_prev = 0;
        sm.prev_last = 0;
        WorkItem none;
        none.kind = 0;
        const long long g = static_cast<long long>(atomicAdd(&a.ctrl->ticket_head, 1ull));
        sm.w[0] = resolve_blocking<Tr>(a, g, none);
        if (sm.w[0].kind == 1) issue_tile_load<Tr>(a, sm.w[0], sm, 0);
        if (!a.ordered) g_ahead = static_cast<long long>(atomicAdd(&a.ctrl->ticket_head, 1ull));
    }
    __syncthreads();
    if (a.profile && tid == 0) sm.tm[0] += prof_clock() - t_wait;
    int b = 0;
    if (Tr::PF && sm.w[0].kind == 1 && sm.w[0].full) pending |= 1u;
    bool aborted = false;
    // The current work item lives in sm.w[0], the next one in sm.w[1].
    while (sm.w[0].kind == 1) {
        if (tid == 0) {
            // Claim the next ticket now; prefetch its tile if its task is known.
            const long long th = a.profile ? prof_clock() : 0;
            long long g;
            if (a.ordered) {
                g = static_cast<long long>(atomicAdd(&a.ctrl->ticket_head, 1ull));
            } else {
                g = g_ahead;
                g_ahead = static_cast<long long>(atomicAdd(&a.ctrl->ticket_head, 1ull));
                if (a.profile) sm.tm[11] += prof_clock() - th;
            }
            sm.next_ticket = g;
            const long long tr = a.profile ? prof_clock() : 0;
            sm.w[1] = try_resolve<Tr>(a, g, sm.w[0]);
            const long long ti = a.profile ? prof_clock() : 0;
            if (sm.w[1].kind == 1) issue_tile_load<Tr>(a, sm.w[1], sm, b ^ 1);
            if (a.profile) {
                const long long now = prof_clock();
                sm.tm[13] += now - th;
                sm.tm[24] += ti - tr;
                sm.tm[25] += now - ti;
            }
        }
        const int r = partition_tile<Tr>(a, sm.w[0], sm.w[1], sm, b, phases);
        if (r != -1) pending &= ~(1u << b);  // -1: the copy into buffer b was never seen to land
        if (Tr::PF && sm.w[1].kind == 1 && sm.w[1].full) pending |= 1u << (b ^ 1);  // written before the tile's barriers
        if (r < 0) {
            aborted = true;
            break;
        }
        if (sm.prev_last) {
            const long long t6 = a.profile ? prof_clock() : 0;
            finish_task<Tr>(a, sm.wf, sm);
            if (a.profile && tid == 0) sm.tm[6] += prof_clock() - t6;
        }
        if (sm.w[1].kind == 0) {
            // About to wait for work: release the last written tile first, as
            // the work waited for may be its task's children.
            flush_release<Tr>(a, sm);
            const long long t0w = a.profile ? prof_clock() : 0;
            __syncthreads();
            if (tid == 0) {
                sm.w[1] = resolve_blocking<Tr>(a, sm.next_ticket, sm.w[0]);
                if (sm.w[1].kind == 1) issue_tile_load<Tr>(a, sm.w[1], sm, b ^ 1);
            }
            __syncthreads();
            if (Tr::PF && sm.w[1].kind == 1 && sm.w[1].full) pending |= 1u << (b ^ 1);
            if (a.profile && tid == 0) sm.tm[0] += prof_clock() - t0w;
        }
        __syncthreads();
        if (tid == 0) sm.w[0] = sm.w[1];
        __syncthreads();
        b ^= 1;
    }
    if (!aborted) flush_release<Tr>(a, sm);
    // Never leave while a bulk copy may still be writing this CTA's shared
    // memory: the next CTA on this SM could receive it.  `pending` and
    // `phases` are the same in every thread (both change only at points the
    // whole CTA passes together), so every thread waits for the same copies.
    // A copy that was issued always lands, within microseconds; the wait's
    // floor of kDrainFloorNs keeps a small QS_OPT_WAIT_LIMIT_NS from cutting
    // it short (a timed-out drain records QS_ERR_TIMEOUT like any wait).
    const uint64_t drain_ns = a.wait_limit_ns > kDrainFloorNs ? a.wait_limit_ns : kDrainFloorNs;
    for (int i = 0; i < 2; ++i)
        if ((pending >> i) & 1u) mbar_wait_bounded(&sm.bar[i], (phases >> i) & 1u, a.ctrl, drain_ns);
    __syncthreads();
    if (a.profile && tid == 0)
        for (int i = 0; i < kProfSlots; ++i) atomicAdd(&a.ctrl->cycles[i], static_cast<unsigned long long>(sm.tm[i]));
    if (aborted) return;
    // Clean exit: every task is finished, so no CTA reads the look-back words
    // or the ticket owners any more; clear this CTA's share for the next call.
    // (A partition-only call's CTAs leave while others may still read the
    // look-back words; the host clears the words it used before the next call.)
    if (!a.partition_only && ld_relaxed_s32(&a.ctrl->status) == 0) {
        const unsigned long long used = ld_relaxed_u64(&a.ctrl->pool_cursor);
        const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * Tr::DT;
        for (unsigned long long i = blockIdx.x * Tr::DT + tid; i < used; i += stride) {
            a.pool[i] = 0;
            a.owner[i] = 0;
        }
        if (tid == 0) atomicAdd(&a.ctrl->exited, 1ull);
    }
}

// ---------------------------------------------------------------------------
// Setup: one CTA resets the control block and seeds the root task.
// ---------------------------------------------------------------------------
template <class Tr>
__global__ void __launch_bounds__(kThreads) setup_kernel(Args<typename Tr::K, typename Tr::V> a)
{
    using K = typename Tr::K;
    __shared__ NewTask nt;
    __shared__ int ok;
    Ctrl *c = a.ctrl;
    const int tid = threadIdx.x;
    if (tid == 0) {
        c->ticket_head = 0;
        c->n_tasks = c->pool_cursor = 0;
        c->pending = 0;
        c->n_large = c->n_small = 0;
        c->claim_large = c->claim_small = 0;
        // An error of the previous call that the host has not read yet is
        // kept (asynchronous calls report it at the next synchronisation).
        if (c->status != 0 && c->sticky == 0) {
            c->sticky = c->status;
            c->sticky_info = c->info;
        }
        c->status = 0;
        c->info = 0;
        c->part_tasks = c->part_keys = c->leaf_parts = c->leaf_keys = c->copy_keys = c->max_depth = 0;
        c->mid_parts = c->mid_keys = 0;
        c->lt_result = 0;
        c->exited = 0;
        for (int i = 0; i < kProfSlots; ++i) c->cycles[i] = 0;
        ok = 0;
        __threadfence();
    }
    __syncthreads();
    if (a.seg_off) {
        // Segmented sort: setup_segments_kernel seeds the work.
    } else if (a.partition_only || a.n > a.leaf_max) {
        uint64_t pbits = a.pivot_bits;
        if (!a.partition_only && tid < 32) pbits = sample_median<K>(a.keys[0], 0, a.n, 0x51ED5EEDull);
        if (tid == 0) {
            ok = alloc_task<Tr>(a, 0, a.n, 0, pbits, kModeLess, 0, nt);
            if (ok) c->pending = 1;
        }
        __syncthreads();
        if (ok) publish_task(a.owner, nt);
    } else if (a.n > 1) {
        if (tid == 0) push_leaf<Tr>(a, 0, a.n, 0);
    }
}

// ---------------------------------------------------------------------------
// Segmented sort setup: one lane per segment for the leaves, one warp per
// partition task.  A segment of at most leaf_max
// keys goes straight to the leaf list; a larger one becomes a partition task
// with a sampled pivot.  Offsets are checked on the device (0 <= off[i] <=
// off[i+1] <= n); a bad table records QS_ERR_INVALID_ARG.
// ---------------------------------------------------------------------------
template <class Tr>
__global__ void __launch_bounds__(kThreads) setup_segments_kernel(Args<typename Tr::K, typename Tr::V> a)
{
    using K = typename Tr::K;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const long long warp = (static_cast<long long>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
    const long long nwarps = (static_cast<long long>(gridDim.x) * kThreads) >> 5;
    const int src = a.seg_src;
    // 32 segments per warp step, one per lane: the leaves of a step are listed
    // with one reservation per side (a step of tiny segments costs a few
    // atomics, not a few per segment).
    for (long long s0 = warp * 32; s0 < a.nseg; s0 += nwarps * 32) {
        const long long i = s0 + lane;
        int kind = 0;  // 0 nothing, 1 small leaf, 2 large leaf, 3 partition task
        int64_t off = 0, len = 0;
        if (i < a.nseg) {
            off = a.seg_off[i];
            const int64_t end = a.seg_off[i + 1];
            if (off < 0 || end < off || end > a.n) {
                set_error(a.ctrl, -1, static_cast<int>(i));
            } else {
                len = end - off;
                if (len <= 1) {  // already sorted; from scratch it only has to move home
                    if (len == 1 && src) {
                        a.keys[0][off] = a.keys[1][off];
                        if constexpr (Tr::KV) a.vals[0][off] = a.vals[1][off];
                    }
                } else if (len <= a.leaf_max) {
                    kind = len <= a.small_max ? 1 : 2;
                } else {
                    kind = 3;
                }
            }
        }
        const unsigned sm_mask = __ballot_sync(0xffffffffu, kind == 1);
        const unsigned lg_mask = __ballot_sync(0xffffffffu, kind == 2);
        long long base_s = -1, base_l = -1;
        if (lane == 0) {
            if (sm_mask) base_s = reserve_leaves<Tr>(a, __popc(sm_mask), true);
            if (lg_mask) base_l = reserve_leaves<Tr>(a, __popc(lg_mask), false);
        }
        base_s = __shfl_sync(0xffffffffu, base_s, 0);
        base_l = __shfl_sync(0xffffffffu, base_l, 0);
        if ((kind == 1 && base_s >= 0) || (kind == 2 && base_l >= 0)) {
            Leaf l;
            l.off = off;
            l.len = static_cast<int32_t>(len);
            l.flags = src ? kLeafScratch : 0;
            // the small side grows downward from the end of the list
            const long long at = kind == 1 ? base_s - __popc(sm_mask & below) : base_l + __popc(lg_mask & below);
            a.leaves[at] = l;
        }
        unsigned long long nk = (kind == 1 || kind == 2) ? static_cast<unsigned long long>(len) : 0ull;
        unsigned long long np = (kind == 1 || kind == 2) ? 1ull : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nk += __shfl_xor_sync(0xffffffffu, nk, o);
            np += __shfl_xor_sync(0xffffffffu, np, o);
        }
        if (lane == 0 && np) {
            atomicAdd(&a.ctrl->leaf_parts, np);
            atomicAdd(&a.ctrl->leaf_keys, nk);
        }
    }
    // Partition tasks, one warp each (they are few; each needs a pivot sample).
    for (long long i = warp; i < a.nseg; i += nwarps) {
        const int64_t off = a.seg_off[i], end = a.seg_off[i + 1];
        if (off < 0 || end < off || end > a.n || end - off <= a.leaf_max) continue;
        const int64_t len = end - off;
        const uint64_t pbits =
            sample_median<K>(a.keys[src], off, len, static_cast<uint64_t>(off) * 0x9E3779B97F4A7C15ull + len);
        NewTask nt;
        int ok = 0;
        if (lane == 0) {
            ok = alloc_task<Tr>(a, off, len, src, pbits, kModeLess, 0, nt);
            if (ok) atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctrl->pending), 1ull);
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) continue;
        nt.id = __shfl_sync(0xffffffffu, nt.id, 0);
        nt.g0 = __shfl_sync(0xffffffffu, nt.g0, 0);
        nt.ntiles = __shfl_sync(0xffffffffu, nt.ntiles, 0);
        publish_task(a.owner, nt, lane, 32);
    }
}

}  // namespace qs
