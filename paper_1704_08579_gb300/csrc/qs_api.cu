// C-ABI of libqs.so: argument checks, the per-device workspace, and dispatch
// to the per-kind launchers.  Every entry point is declared and documented in
// include/qs.h.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qs.h"
#include "qs_internal.h"

namespace qs {
namespace {

thread_local std::string t_error;
thread_local qs_stats t_stats;

std::atomic<int> g_profile{0};  // 1: CUDA events around kernels; 2: also in-kernel cycle counters
std::atomic<int64_t> g_wait_limit_ns{2000000000ll};
std::atomic<int64_t> g_task_cap{0};
std::atomic<int64_t> g_driver_ctas{0};
std::atomic<int64_t> g_leaf_max{0};   // 0 = the kind's default (one CTA's shared memory)
std::atomic<int64_t> g_small_max{0};  // 0 = the kind's compiled maximum
std::atomic<int64_t> g_driver_items{0};  // 0 = the kind's default partition tile
std::atomic<int> g_ordered{0};  // 1 = the sort's partitions place tiles in input order too
std::atomic<int> g_sync{0};     // 1 = sorts return only after their work has finished
std::atomic<int> g_bucket_levels{0};  // learned / sampled sorts: 1 or 2 bucket levels, 0 = the default (2)

constexpr int64_t kMaxN = 1ll << 38;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(QS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct Workspace {
    std::mutex mu;
    std::mutex host_mu;  // host-buffer sorts: one at a time (they share the staging area)
    bool init = false;
    int sms = 0;
    int occ[3][4] = {};  // per kind: driver (wide tile), leaf, driver (narrow tile), driver (register tile)
    void *scratch_k = nullptr, *scratch_v = nullptr;
    size_t scratch_k_bytes = 0, scratch_v_bytes = 0;
    void *stage_k = nullptr, *stage_v = nullptr;
    size_t stage_k_bytes = 0, stage_v_bytes = 0;
    Task *tasks = nullptr;
    int64_t task_cap = 0;
    unsigned long long *pool = nullptr;
    int32_t *owner = nullptr;
    int64_t pool_cap = 0;
    Leaf *leaves = nullptr;
    int64_t leaf_cap = 0;
    Ctrl *ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;
    bool dirty = true;  // look-back words / ticket owners must be cleared before use
    int64_t dirty_words = 0;  // else: the first dirty_words of them (left by a partition-only call)
    cudaEvent_t ev[6] = {};
    // Ordering of calls on this workspace: every call waits (on its own
    // stream) for `done`, recorded after the previous call's last operation,
    // so calls on different streams never overlap on the shared buffers.
    cudaEvent_t done = nullptr;
    bool done_recorded = false;
    bool unreported = false;  // the last call's status (copied to h_ctrl) has not been examined
    int64_t last_grid_driver = 0, last_grid_leaf = 0, last_n = 0, last_kind = 0;
    cudaStream_t capture = nullptr;  // private stream used to capture CUDA graphs
    void *aux = nullptr;                   // learned-splitter / bucket state
    void *cnt2 = nullptr;                  // second bucket level: per-chunk sub-bucket counts
    size_t cnt2_bytes = 0;
    LearnedState *h_learned = nullptr;     // pinned copy of its state
    struct Graph {
        std::string key;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<Graph> graphs;  // segmented sorts, most recent last
};

void drop_graphs(Workspace &w)
{
    for (auto &g : w.graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    w.graphs.clear();
}

constexpr int kMaxDevices = 64;
Workspace *g_ws[kMaxDevices] = {};
std::mutex g_ws_mu;

Workspace *workspace_for(int dev)
{
    std::lock_guard<std::mutex> g(g_ws_mu);
    if (!g_ws[dev]) g_ws[dev] = new Workspace();
    return g_ws[dev];
}

KernelLimits limits_of(int kind)
{
    return kind == QS_KIND_I32 ? limits_i32() : kind == QS_KIND_F64 ? limits_f64() : limits_kv();
}

int occupancy_of(int kind, int which, int *bps)
{
    return kind == QS_KIND_I32 ? occupancy_i32(which, bps)
           : kind == QS_KIND_F64 ? occupancy_f64(which, bps)
                                 : occupancy_kv(which, bps);
}

// Grows a device buffer to at least `bytes`; contents are not preserved.
int grow(void **p, size_t *have, size_t bytes, const char *what)
{
    if (*have >= bytes && *p) return QS_OK;
    if (*p) {
        cudaError_t e = cudaFree(*p);
        *p = nullptr;
        *have = 0;
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    cudaError_t e = cudaMalloc(p, bytes < 256 ? 256 : bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(QS_ERR_OOM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    *have = bytes < 256 ? 256 : bytes;
    return QS_OK;
}

int ws_init(Workspace &w)
{
    if (w.init) return QS_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&w.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    for (int k = 0; k < 3; ++k)
        for (int which = 0; which < 4; ++which) {
            e = static_cast<cudaError_t>(occupancy_of(k, which, &w.occ[k][which]));
            if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
            if (w.occ[k][which] < 1) return fail(QS_ERR_INTERNAL, "kernel cannot be resident (kind %d)", k);
        }
    e = cudaMalloc(&w.ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) return fail(QS_ERR_OOM, "cudaMalloc(ctrl): %s", cudaGetErrorString(e));
    e = cudaMallocHost(&w.h_ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) return fail(QS_ERR_OOM, "cudaMallocHost(ctrl): %s", cudaGetErrorString(e));
    for (auto &ev : w.ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
    e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    w.done_recorded = false;
    w.unreported = false;
    w.init = true;
    return QS_OK;
}

struct Needs {
    size_t key_bytes, val_bytes;
    int64_t task_cap, pool_cap, leaf_cap;
};

// Occupancy slot of the partition tile variant selected by `items` (keys per thread).
int tile_variant(int kind, int items)
{
    const KernelLimits l = limits_of(kind);
    if (l.items_xwide && items == l.items_xwide) return 3;
    return items == l.items_narrow ? 2 : 0;
}

int64_t leaf_max_of(int kind)
{
    const KernelLimits l = limits_of(kind);
    const int64_t want = g_leaf_max.load();
    if (want <= 0) return l.leaf_default;
    return want < l.leaf_max ? want : l.leaf_max;
}

int64_t small_max_of(int kind)
{
    const int64_t compiled = limits_of(kind).small_max, want = g_small_max.load();
    const int64_t v = want > 0 && want < compiled ? want : compiled;
    return v < leaf_max_of(kind) ? v : leaf_max_of(kind);
}

Needs needs_for(int64_t n, int kind, int64_t nseg = 0)
{
    const KernelLimits l = limits_of(kind);
    Needs r;
    r.key_bytes = static_cast<size_t>(n) * (kind == QS_KIND_F64 ? 8 : 4);
    r.val_bytes = kind == QS_KIND_KV ? static_cast<size_t>(n) * 4 : 0;
    const int64_t cap_override = g_task_cap.load();
    r.task_cap = cap_override > 0 ? cap_override : 8 * (n / leaf_max_of(kind)) + 1024 + nseg;
    r.pool_cap = 64 * (n / l.tile + 1) + 2 * r.task_cap + 4096;
    r.leaf_cap = 4 * r.task_cap + n / kCopyChunk + 1024 + nseg;
    return r;
}

int ws_ensure(Workspace &w, int64_t n, int kind, int64_t nseg = 0)
{
    int rc = ws_init(w);
    if (rc) return rc;
    const Needs nd = needs_for(n, kind, nseg);
    const void *before[] = {w.scratch_k, w.scratch_v, w.tasks, w.pool, w.owner, w.leaves};
    if ((rc = grow(&w.scratch_k, &w.scratch_k_bytes, nd.key_bytes, "scratch keys"))) return rc;
    if (nd.val_bytes && (rc = grow(&w.scratch_v, &w.scratch_v_bytes, nd.val_bytes, "scratch values"))) return rc;
    const bool override_cap = g_task_cap.load() > 0;
    if (w.task_cap < nd.task_cap || (override_cap && w.task_cap != nd.task_cap)) {
        if (w.tasks) cudaFree(w.tasks);
        w.tasks = nullptr;
        w.task_cap = 0;
        size_t have_t = 0;
        if ((rc = grow(reinterpret_cast<void **>(&w.tasks), &have_t, nd.task_cap * sizeof(Task), "tasks"))) return rc;
        w.task_cap = nd.task_cap;
    }
    if (w.pool_cap < nd.pool_cap) {
        // Look-back words and ticket owners are sized together.
        if (w.pool) cudaFree(w.pool);
        if (w.owner) cudaFree(w.owner);
        w.pool = nullptr;
        w.owner = nullptr;
        w.pool_cap = 0;
        size_t have_p = 0, have_o = 0;
        if ((rc = grow(reinterpret_cast<void **>(&w.pool), &have_p, nd.pool_cap * 8, "look-back words"))) return rc;
        if ((rc = grow(reinterpret_cast<void **>(&w.owner), &have_o, nd.pool_cap * 4, "ticket owners"))) return rc;
        w.pool_cap = nd.pool_cap;
        w.dirty = true;
    }
    if (w.leaf_cap < nd.leaf_cap) {
        size_t have = w.leaves ? static_cast<size_t>(w.leaf_cap) * sizeof(Leaf) : 0;
        if ((rc = grow(reinterpret_cast<void **>(&w.leaves), &have, nd.leaf_cap * sizeof(Leaf), "leaf list"))) return rc;
        w.leaf_cap = nd.leaf_cap;
    }
    const void *after[] = {w.scratch_k, w.scratch_v, w.tasks, w.pool, w.owner, w.leaves};
    for (int i = 0; i < 6; ++i)
        if (before[i] != after[i]) {
            drop_graphs(w);  // captured graphs point at the old buffers
            break;
        }
    return QS_OK;
}

void ws_free(Workspace &w)
{
    if (!w.init) return;
    cudaDeviceSynchronize();
    drop_graphs(w);
    if (w.capture) cudaStreamDestroy(w.capture);
    w.capture = nullptr;
    void *bufs[] = {w.scratch_k, w.scratch_v, w.stage_k, w.stage_v, w.tasks, w.owner, w.pool, w.leaves, w.ctrl, w.aux, w.cnt2};
    if (w.h_learned) cudaFreeHost(w.h_learned);
    w.aux = nullptr;
    w.cnt2 = nullptr;
    w.cnt2_bytes = 0;
    w.h_learned = nullptr;
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (w.h_ctrl) cudaFreeHost(w.h_ctrl);
    for (auto &ev : w.ev)
        if (ev) cudaEventDestroy(ev);
    if (w.done) cudaEventDestroy(w.done);
    w.done = nullptr;
    w.done_recorded = false;
    w.unreported = false;
    w.scratch_k = w.scratch_v = w.stage_k = w.stage_v = nullptr;
    w.scratch_k_bytes = w.scratch_v_bytes = w.stage_k_bytes = w.stage_v_bytes = 0;
    w.tasks = nullptr;
    w.owner = nullptr;
    w.pool = nullptr;
    w.leaves = nullptr;
    w.ctrl = nullptr;
    w.h_ctrl = nullptr;
    w.task_cap = w.pool_cap = w.leaf_cap = 0;
    for (auto &ev : w.ev) ev = nullptr;
    w.dirty = true;
    w.init = false;
}

template <class K>
int phase_of(const void *p)
{
    return static_cast<int>((reinterpret_cast<uintptr_t>(p) / sizeof(K)) % (16 / sizeof(K)));
}

const char *status_text(int s)
{
    switch (s) {
    case QS_ERR_TIMEOUT: return "a device-side wait ran out (QS_OPT_WAIT_LIMIT_NS)";
    case QS_ERR_CAPACITY: return "device task/look-back/leaf capacity exceeded";
    case QS_ERR_INTERNAL: return "recursion deeper than the supported limit, or a device index check failed";
    default: return "device error";
    }
}

// Kernel arguments for a call on workspace w.
template <class K>
Args<K, int32_t> make_args(Workspace &w, int kind, K *keys, int32_t *vals, int64_t n)
{
    Args<K, int32_t> a;
    std::memset(&a, 0, sizeof(a));
    a.keys[0] = keys;
    a.keys[1] = static_cast<K *>(w.scratch_k);
    a.vals[0] = vals;
    a.vals[1] = kind == QS_KIND_KV ? static_cast<int32_t *>(w.scratch_v) : nullptr;
    for (int b = 0; b < 2; ++b) {
        a.key_phase[b] = phase_of<K>(a.keys[b]);
        a.val_vec[b] = a.vals[b] ? (phase_of<int32_t>(a.vals[b]) == a.key_phase[b]) : 1;
    }
    a.n = n;
    a.tasks = w.tasks;
    a.owner = w.owner;
    a.pool = w.pool;
    a.leaves = w.leaves;
    a.ctrl = w.ctrl;
    a.task_cap = w.task_cap;
    a.pool_cap = w.pool_cap;
    a.leaf_cap = w.leaf_cap;
    a.leaf_max = leaf_max_of(kind);
    a.small_max = small_max_of(kind);
    a.wait_limit_ns = static_cast<uint64_t>(g_wait_limit_ns.load());
    a.ordered = g_ordered.load();
    a.profile = g_profile.load() >= 2 ? 1 : 0;
    a.okeys = a.keys[0];
    a.ovals = a.vals[0];
    a.out_separate = 0;
    return a;
}

// Clears the look-back words and ticket owners a previous call left set.
cudaError_t clear_dirty(Workspace &w, cudaStream_t s)
{
    const int64_t words = w.dirty ? w.pool_cap : (w.dirty_words < w.pool_cap ? w.dirty_words : w.pool_cap);
    cudaError_t e = cudaSuccess;
    if (words > 0) {
        e = cudaMemsetAsync(w.pool, 0, static_cast<size_t>(words) * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.owner, 0, static_cast<size_t>(words) * 4, s);
    }
    if (e == cudaSuccess) {
        w.dirty = false;
        w.dirty_words = 0;
    }
    return e;
}

// Ordering of the calls that share a workspace: `s` waits for the last
// operation of the previous call, whatever stream it was issued on.
cudaError_t order_after_previous(Workspace &w, cudaStream_t s)
{
    return w.done_recorded ? cudaStreamWaitEvent(s, w.done, 0) : cudaSuccess;
}

cudaError_t mark_done(Workspace &w, cudaStream_t s)
{
    const cudaError_t e = cudaEventRecord(w.done, s);
    if (e == cudaSuccess) w.done_recorded = true;
    return e;
}

// Device counters of the last finished call (read from the control block it
// copied back) into this thread's statistics.
void stats_from_ctrl(const Workspace &w)
{
    const Ctrl &c = *w.h_ctrl;
    t_stats.n = w.last_n;
    t_stats.kind = w.last_kind;
    t_stats.part_tasks = static_cast<int64_t>(c.part_tasks);
    t_stats.part_keys = static_cast<int64_t>(c.part_keys);
    t_stats.leaf_parts = static_cast<int64_t>(c.leaf_parts);
    t_stats.leaf_keys = static_cast<int64_t>(c.leaf_keys);
    t_stats.copy_keys = static_cast<int64_t>(c.copy_keys);
    t_stats.max_depth = static_cast<int64_t>(c.max_depth);
    t_stats.mid_parts = static_cast<int64_t>(c.mid_parts);
    t_stats.mid_keys = static_cast<int64_t>(c.mid_keys);
    t_stats.lookback_words = static_cast<int64_t>(c.pool_cursor);
    t_stats.grid_driver = w.last_grid_driver;
    t_stats.grid_leaf = w.last_grid_leaf;
    for (int i = 0; i < kProfSlots; ++i) t_stats.driver_cycles[i] = static_cast<int64_t>(c.cycles[i]);
}

// Examines the status that the last call copied back (its work has
// finished).  Returns QS_OK, or the first device-side error not reported yet
// -- an earlier asynchronous call's (kept in the sticky word by the setup
// kernel of the calls after it) or the last call's -- and clears it on the
// device, so each failure is reported once.
int report_status(Workspace &w, cudaStream_t s, bool earlier_call = false)
{
    static_assert(offsetof(Ctrl, sticky_info) == offsetof(Ctrl, status) + 3 * sizeof(int),
                  "status, info, sticky, sticky_info are contiguous");
    w.unreported = false;
    Ctrl &c = *w.h_ctrl;
    const bool sticky = c.sticky != 0;
    const int err = sticky ? c.sticky : c.status;
    if (err == 0) return QS_OK;
    const int info = sticky ? c.sticky_info : c.info;
    const bool earlier = sticky || earlier_call;
    c.status = c.sticky = 0;
    w.dirty = true;  // look-back words and ticket owners are cleared before the next call
    cudaError_t e = cudaMemsetAsync(&w.ctrl->status, 0, 4 * sizeof(int), s);
    if (e == cudaSuccess) e = mark_done(w, s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the status word");
    return fail(err, "%s%s (code %d, detail %d)", earlier ? "an earlier asynchronous call failed: " : "",
                status_text(err), err, info);
}

// Before a call enqueues work: an earlier asynchronous call that has finished
// with an error is reported now, and the new call does nothing.
int check_earlier(Workspace &w, cudaStream_t s)
{
    if (!w.unreported || !w.done_recorded) return QS_OK;
    const cudaError_t q = cudaEventQuery(w.done);
    if (q == cudaErrorNotReady) {
        if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
        return QS_OK;  // still running: its error, if any, is kept on the device
    }
    if (q != cudaSuccess) return cuda_fail(q, "cudaEventQuery");
    stats_from_ctrl(w);
    return report_status(w, s, true);
}

// Runs one sort (partition_only = 0) or partition (1) of kind `kind` on the
// current device.  keys/vals are device pointers.  A partition, a call with
// profiling on, a call with QS_OPT_SYNC = 1 and a call with force_sync
// return after the work has finished; other sorts return once it is
// enqueued (asynchronous: the status is read by qs_sync_status or reported
// by the next call).
template <class K>
int64_t run(int kind, K *keys, int32_t *vals, int64_t n, uint64_t pivot_bits, int partition_only,
            qs_stream_t stream, const int64_t *seg_off = nullptr, int64_t nseg = 0, bool force_sync = false,
            K *out_keys = nullptr, int32_t *out_vals = nullptr)
{
    t_error.clear();
    std::memset(&t_stats, 0, sizeof(t_stats));
    t_stats.n = n;
    t_stats.kind = kind;
    if (n < 0 || n > kMaxN) return fail(QS_ERR_INVALID_ARG, "n = %lld out of range [0, 2^38]", (long long)n);
    if (nseg < 0 || nseg > (1ll << 31)) return fail(QS_ERR_INVALID_ARG, "nseg = %lld out of range", (long long)nseg);
    if (nseg > 0 && !seg_off) return fail(QS_ERR_INVALID_ARG, "null offsets pointer");
    if (seg_off && reinterpret_cast<uintptr_t>(seg_off) % 8) return fail(QS_ERR_ALIGN, "offsets not aligned to 8 bytes");
    if (seg_off && nseg == 0) return QS_OK;
    if (n == 0 || (n == 1 && !partition_only)) {
        if (partition_only) return 0;
        return QS_OK;
    }
    if (!keys) return fail(QS_ERR_INVALID_ARG, "null key pointer");
    if (kind == QS_KIND_KV && !vals) return fail(QS_ERR_INVALID_ARG, "null value pointer");
    if (reinterpret_cast<uintptr_t>(keys) % sizeof(K)) return fail(QS_ERR_ALIGN, "keys not aligned to %zu bytes", sizeof(K));
    if (vals && reinterpret_cast<uintptr_t>(vals) % 4) return fail(QS_ERR_ALIGN, "values not aligned to 4 bytes");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(QS_ERR_INVALID_ARG, "device %d out of range", dev);
    Workspace &w = *workspace_for(dev);
    std::lock_guard<std::mutex> guard(w.mu);
    int rc = ws_ensure(w, n, kind, nseg);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((rc = check_earlier(w, s))) return rc;
    if ((e = order_after_previous(w, s)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if ((e = clear_dirty(w, s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    Args<K, int32_t> a = make_args<K>(w, kind, keys, vals, n);
    if (out_keys) {  // the sorted result goes to a separate (mapped host) array
        a.okeys = out_keys;
        a.ovals = out_vals;
        a.out_separate = 1;
    }
    a.pivot_bits = pivot_bits;
    a.partition_only = partition_only;
    if (partition_only) a.ordered = 1;
    a.seg_off = seg_off;
    a.nseg = nseg;

    LaunchCfg cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.stream = s;
    const int64_t ctas = g_driver_ctas.load();
    cfg.items = static_cast<int>(g_driver_items.load());
    if (cfg.items == 0) cfg.items = partition_only ? limits_of(kind).items_default_part : limits_of(kind).items_default;
    cfg.grid_driver = ctas > 0 ? static_cast<int>(ctas) : w.sms * w.occ[kind][tile_variant(kind, cfg.items)];
    cfg.grid_leaf = ctas > 0 ? static_cast<int>(ctas) : w.sms * w.occ[kind][1];
    cfg.profile = g_profile.load();
    for (int i = 0; i < 6; ++i) cfg.ev[i] = w.ev[i];

    auto enqueue = [&](cudaStream_t st) -> cudaError_t {
        LaunchCfg c2 = cfg;
        c2.stream = st;
        int le = 0;
        if constexpr (sizeof(K) == 8)
            le = launch_f64(a, c2);
        else
            le = kind == QS_KIND_I32 ? launch_i32(a, c2) : launch_kv(a, c2);
        if (le != cudaSuccess) return static_cast<cudaError_t>(le);
        return cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    };
    if (seg_off) {
        // Segmented sorts replay one CUDA graph (setup, persistent partition
        // kernel, leaf kernel, status read-back) per argument set.
        cfg.profile = 0;
        char key[320];
        snprintf(key, sizeof(key), "%d:%p:%p:%p:%lld:%lld:%lld:%lld:%d:%d:%d:%d:%llu", kind, (void *)keys,
                 (void *)vals, (const void *)seg_off, (long long)n, (long long)nseg, (long long)a.leaf_max,
                 (long long)a.small_max, cfg.grid_driver, cfg.grid_leaf, cfg.items, a.ordered,
                 (unsigned long long)a.wait_limit_ns);
        cudaGraphExec_t exec = nullptr;
        for (auto &g : w.graphs)
            if (g.key == key) exec = g.exec;
        if (!exec) {
            if (!w.capture && (e = cudaStreamCreateWithFlags(&w.capture, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate");
            cudaGraph_t graph = nullptr;
            if ((e = cudaStreamBeginCapture(w.capture, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamBeginCapture");
            const cudaError_t le = enqueue(w.capture);
            e = cudaStreamEndCapture(w.capture, &graph);
            if (le != cudaSuccess) return cuda_fail(le, "kernel launch (capture)");
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            if (w.graphs.size() >= 8) {
                cudaGraphExecDestroy(w.graphs.front().exec);
                w.graphs.erase(w.graphs.begin());
            }
            w.graphs.push_back(Workspace::Graph{key, exec});
        }
        if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    } else {
        if ((e = enqueue(s)) != cudaSuccess) return cuda_fail(e, "kernel launch");
    }
    if ((e = mark_done(w, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    w.unreported = true;
    w.last_n = n;
    w.last_kind = kind;
    w.last_grid_driver = cfg.grid_driver;
    w.last_grid_leaf = cfg.grid_leaf;
    t_stats.grid_driver = cfg.grid_driver;
    t_stats.grid_leaf = cfg.grid_leaf;
    if (!(partition_only || force_sync || cfg.profile || g_sync.load())) return QS_OK;

    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    stats_from_ctrl(w);
    const unsigned long long lt = w.h_ctrl->lt_result;
    if ((rc = report_status(w, s))) return rc;
    if (partition_only) {
        // Its CTAs left without clearing the look-back words they used.
        w.dirty_words = static_cast<int64_t>(w.h_ctrl->pool_cursor);
        // The split is known.  The lower side was written in place; move the
        // upper side, [lt, n), back from scratch into the caller's arrays.
        if (cfg.profile) cudaEventRecord(w.ev[4], s);
        const size_t hi = static_cast<size_t>(n) - static_cast<size_t>(lt);
        if (lt > static_cast<unsigned long long>(n)) return fail(QS_ERR_INTERNAL, "split beyond the array");
        if (hi && (e = cudaMemcpyAsync(keys + lt, static_cast<K *>(w.scratch_k) + lt, hi * sizeof(K),
                                       cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(copy-back)");
        if (hi && kind == QS_KIND_KV &&
            (e = cudaMemcpyAsync(vals + lt, static_cast<int32_t *>(w.scratch_v) + lt, hi * 4, cudaMemcpyDeviceToDevice,
                                 s)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(copy-back)");
        if (cfg.profile) cudaEventRecord(w.ev[5], s);
        if ((e = mark_done(w, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    if (cfg.profile) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, w.ev[1], w.ev[2]) == cudaSuccess) t_stats.ms_driver = ms;
        if (!partition_only && cudaEventElapsedTime(&ms, w.ev[2], w.ev[3]) == cudaSuccess) t_stats.ms_leaf = ms;
        if (partition_only && cudaEventElapsedTime(&ms, w.ev[4], w.ev[5]) == cudaSuccess) t_stats.ms_copy = ms;
        if (cudaEventElapsedTime(&ms, w.ev[0], partition_only ? w.ev[5] : w.ev[3]) == cudaSuccess) t_stats.ms_total = ms;
    }
    return partition_only ? static_cast<int64_t>(lt) : QS_OK;
}

// Device address of a host buffer the GPU can write (pinned memory mapped
// into the device's address space), or nullptr (pageable memory).
template <class T>
T *mapped_device_ptr(T *h)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    if (reinterpret_cast<uintptr_t>(at.devicePointer) % sizeof(T)) return nullptr;
    return static_cast<T *>(at.devicePointer);
}

// Host-buffer sort: the keys (and values) are copied into a device staging
// area and sorted there.  When the host buffers are mapped pinned memory, the
// leaf kernel writes every sorted part straight into them, so the copy back
// overlaps the leaf sorts instead of following them; otherwise the result is
// copied back after the sort.
template <class K>
int run_host(int kind, K *h_keys, int32_t *h_vals, int64_t n, qs_stream_t stream)
{
    t_error.clear();
    if (n < 0 || n > kMaxN) return fail(QS_ERR_INVALID_ARG, "n = %lld out of range [0, 2^38]", (long long)n);
    if (n < 2) return QS_OK;
    if (!h_keys || (kind == QS_KIND_KV && !h_vals)) return fail(QS_ERR_INVALID_ARG, "null host pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(QS_ERR_INVALID_ARG, "device %d out of range", dev);
    Workspace &w = *workspace_for(dev);
    // Held for the whole call: the staging area is filled, sorted and read
    // back before another host-buffer sort on this device may touch it.
    std::lock_guard<std::mutex> host_guard(w.host_mu);
    K *dk = nullptr;
    int32_t *dv = nullptr;
    {
        std::lock_guard<std::mutex> guard(w.mu);
        int rc = ws_init(w);
        if (rc) return rc;
        if ((rc = grow(&w.stage_k, &w.stage_k_bytes, static_cast<size_t>(n) * sizeof(K), "staging keys"))) return rc;
        if (kind == QS_KIND_KV && (rc = grow(&w.stage_v, &w.stage_v_bytes, static_cast<size_t>(n) * 4, "staging values")))
            return rc;
        dk = static_cast<K *>(w.stage_k);
        dv = static_cast<int32_t *>(w.stage_v);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpyAsync(dk, h_keys, static_cast<size_t>(n) * sizeof(K), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(H2D)");
    if (kind == QS_KIND_KV &&
        (e = cudaMemcpyAsync(dv, h_vals, static_cast<size_t>(n) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(H2D)");
    K *mk = mapped_device_ptr(h_keys);
    int32_t *mv = kind == QS_KIND_KV ? mapped_device_ptr(h_vals) : nullptr;
    const bool direct = mk && (kind != QS_KIND_KV || mv);
    const int64_t rc = run<K>(kind, dk, kind == QS_KIND_KV ? dv : nullptr, n, 0, 0, stream, nullptr, 0, true,
                              direct ? mk : nullptr, direct ? mv : nullptr);
    if (rc) return static_cast<int>(rc);
    if (!direct) {
        if ((e = cudaMemcpyAsync(h_keys, dk, static_cast<size_t>(n) * sizeof(K), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(D2H)");
        if (kind == QS_KIND_KV &&
            (e = cudaMemcpyAsync(h_vals, dv, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return QS_OK;
}

constexpr size_t kAuxState = 4096, kAuxSketch = 4096, kAuxSample = 8192, kAuxSpl = 4096;
constexpr size_t kAuxCnt = sizeof(int64_t) * kLearnedBuckets * kMaxBucketCtas, kAuxAct = 4096;
constexpr size_t kAuxSpl2 = sizeof(uint64_t) * kLearnedBuckets2;
constexpr size_t kAuxOff2 = (sizeof(int64_t) * (kLearnedBuckets2 + 1) + 4095) / 4096 * 4096, kAuxCbase = 4096;
constexpr size_t kAuxBytes =
    kAuxState + kAuxSketch + kAuxSample + kAuxSpl + kAuxCnt + kAuxAct + kAuxSpl2 + kAuxOff2 + kAuxCbase;

int aux_ensure(Workspace &w)
{
    if (w.aux) return QS_OK;
    static_assert(sizeof(LearnedState) <= kAuxState, "state fits its slot");
    cudaError_t e = cudaMalloc(&w.aux, kAuxBytes);
    if (e != cudaSuccess) {
        w.aux = nullptr;
        return fail(QS_ERR_OOM, "cudaMalloc(learned state): %s", cudaGetErrorString(e));
    }
    e = cudaMallocHost(&w.h_learned, sizeof(LearnedState));
    if (e != cudaSuccess) return fail(QS_ERR_OOM, "cudaMallocHost(learned state): %s", cudaGetErrorString(e));
    return QS_OK;
}

LearnedPtrs aux_ptrs(Workspace &w)
{
    char *b = static_cast<char *>(w.aux);
    LearnedPtrs p;
    p.st = reinterpret_cast<LearnedState *>(b);
    p.sketch = reinterpret_cast<float *>(b + kAuxState);
    p.sample = b + kAuxState + kAuxSketch;
    p.splitters = b + kAuxState + kAuxSketch + kAuxSample;
    p.cnt = reinterpret_cast<int64_t *>(b + kAuxState + kAuxSketch + kAuxSample + kAuxSpl);
    p.act = reinterpret_cast<float *>(b + kAuxState + kAuxSketch + kAuxSample + kAuxSpl + kAuxCnt);
    char *l2 = b + kAuxState + kAuxSketch + kAuxSample + kAuxSpl + kAuxCnt + kAuxAct;
    p.spl2 = l2;
    p.off2 = reinterpret_cast<int64_t *>(l2 + kAuxSpl2);
    p.cbase = reinterpret_cast<int64_t *>(l2 + kAuxSpl2 + kAuxOff2);
    p.cnt2 = static_cast<int64_t *>(w.cnt2);
    return p;
}

// Sketch (op = kOpSketch), bucket pass by the caller's splitters (kOpBucket)
// or learned / sampled-splitter sort (kOpSortLearned) of i32 or f64 keys.
template <class K>
int run_learned(int kind, K *keys, int64_t n, int op, const float *params, const K *user_spl, int nsplit,
                int64_t *bucket_off_out, float *sketch_out, double *minmax_out, qs_stream_t stream,
                K *sample_out = nullptr)
{
    t_error.clear();
    std::memset(&t_stats, 0, sizeof(t_stats));
    t_stats.n = n;
    t_stats.kind = kind;
    if (n < 0 || n > kMaxN) return fail(QS_ERR_INVALID_ARG, "n = %lld out of range [0, 2^38]", (long long)n);
    if (!keys && n > 0) return fail(QS_ERR_INVALID_ARG, "null key pointer");
    if (reinterpret_cast<uintptr_t>(keys) % sizeof(K)) return fail(QS_ERR_ALIGN, "keys not aligned");
    if (op == kOpSketch && (n < kLearnedSketch || !sketch_out || !minmax_out))
        return fail(QS_ERR_INVALID_ARG, "sketch needs n >= 1024 and output pointers");
    if (op == kOpBucket) {
        if (nsplit < 1 || nsplit > 255 || !user_spl || !bucket_off_out)
            return fail(QS_ERR_INVALID_ARG, "bucket pass needs 1..255 splitters and an offsets array");
        if (n == 0) {  // every bucket starts (and ends) at 0
            const cudaError_t e0 = cudaMemsetAsync(bucket_off_out, 0, sizeof(int64_t) * (nsplit + 2),
                                                   reinterpret_cast<cudaStream_t>(stream));
            return e0 == cudaSuccess ? QS_OK : cuda_fail(e0, "cudaMemsetAsync");
        }
    }
    if (op == kOpSortLearned && n < (1 << 16)) {
        // Too small for 256 buckets to pay: the plain method.
        return static_cast<int>(run<K>(kind, keys, nullptr, n, 0, 0, stream, nullptr, 0, true));
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(QS_ERR_INVALID_ARG, "device %d out of range", dev);
    Workspace &w = *workspace_for(dev);
    std::lock_guard<std::mutex> guard(w.mu);
    const int levels = op == kOpSortLearned ? (g_bucket_levels.load() == 1 ? 1 : 2) : 1;
    const int64_t ctas2 = n / kBucket2Chunk + kLearnedBuckets + 1;  // >= the sum over buckets of ceil(size / chunk)
    int rc = ws_ensure(w, n, kind, levels == 2 ? kLearnedBuckets2 : kLearnedBuckets);
    if (rc) return rc;
    if ((rc = aux_ensure(w))) return rc;
    if (levels == 2 &&
        (rc = grow(&w.cnt2, &w.cnt2_bytes, static_cast<size_t>(ctas2) * kLearnedBuckets * sizeof(int64_t),
                   "second-level bucket counts")))
        return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((rc = check_earlier(w, s))) return rc;
    if ((e = order_after_previous(w, s)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if ((e = clear_dirty(w, s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    Args<K, int32_t> a = make_args<K>(w, kind, keys, nullptr, n);
    LearnedCall lc;
    std::memset(&lc, 0, sizeof(lc));
    lc.p = aux_ptrs(w);
    lc.op = op;
    lc.params = params;
    lc.user_spl = user_spl;
    lc.nsplit = nsplit;
    lc.ctas = w.sms * 4 < kMaxBucketCtas ? w.sms * 4 : kMaxBucketCtas;
    lc.levels = levels;
    lc.ctas2 = static_cast<int>(ctas2);
    lc.bound = 4 * (n / kLearnedBuckets + 1);
    lc.sketch_out = sketch_out;
    lc.minmax_out = minmax_out;
    lc.sample_out = sample_out;
    LaunchCfg cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.stream = s;
    const int64_t ctas = g_driver_ctas.load();
    // The bucket forms' final segmented sort runs the kind's first compiled
    // partition tile (occupancy slot 0) whatever QS_OPT_DRIVER_ITEMS says.
    cfg.items = limits_of(kind).items_wide;
    cfg.grid_driver = ctas > 0 ? static_cast<int>(ctas) : w.sms * w.occ[kind][0];
    cfg.grid_leaf = ctas > 0 ? static_cast<int>(ctas) : w.sms * w.occ[kind][1];
    cfg.profile = g_profile.load();
    for (int i = 0; i < 6; ++i) cfg.ev[i] = w.ev[i];
    int le;
    if constexpr (sizeof(K) == 8)
        le = learned_f64(a, lc, cfg);
    else
        le = learned_i32(a, lc, cfg);
    if (le != cudaSuccess) return cuda_fail(static_cast<cudaError_t>(le), "kernel launch");
    if ((e = cudaMemcpyAsync(w.h_learned, lc.p.st, sizeof(LearnedState), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(status)");
    if ((e = mark_done(w, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    w.unreported = true;
    w.last_n = n;
    w.last_kind = kind;
    w.last_grid_driver = cfg.grid_driver;
    w.last_grid_leaf = cfg.grid_leaf;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (op == kOpSortLearned) stats_from_ctrl(w);
    if ((rc = report_status(w, s))) return rc;
    const LearnedState &ls = *w.h_learned;
    if (ls.status != 0) return fail(QS_ERR_INTERNAL, "bucket pass index check failed");
    if (op == kOpSortLearned) {
        if (cfg.profile) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, w.ev[1], w.ev[2]) == cudaSuccess) t_stats.ms_driver = ms;
            if (cudaEventElapsedTime(&ms, w.ev[2], w.ev[3]) == cudaSuccess) t_stats.ms_leaf = ms;
        }
    }
    if (op != kOpSketch) {
        t_stats.bucket_max = static_cast<int64_t>(ls.bucket_max);
        t_stats.bucket_over = static_cast<int64_t>(ls.bucket_over);
        t_stats.bucket_dev = static_cast<int64_t>(ls.bucket_dev);
    }
    if (op == kOpBucket) {
        if ((e = cudaMemcpyAsync(keys, w.scratch_k, static_cast<size_t>(n) * sizeof(K), cudaMemcpyDeviceToDevice, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(bucket_off_out, lc.p.st->bucket_off, sizeof(int64_t) * (nsplit + 2),
                                 cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
            (e = mark_done(w, s)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "copy-back");
    }
    return QS_OK;
}

uint64_t bits_i32(int32_t k) { return static_cast<uint64_t>(static_cast<int64_t>(k)); }
uint64_t bits_f64(double k)
{
    if (k == 0.0) k = 0.0;  // a -0.0 pivot splits exactly like +0.0
    uint64_t b;
    std::memcpy(&b, &k, 8);
    return b;
}

}  // namespace

uint64_t option_wait_limit_ns() { return static_cast<uint64_t>(g_wait_limit_ns.load()); }

}  // namespace qs

using namespace qs;

extern "C" {

int64_t qs_partition_i32(int32_t *d_keys, int64_t n, int32_t pivot, qs_stream_t stream)
{
    return run<int32_t>(QS_KIND_I32, d_keys, nullptr, n, bits_i32(pivot), 1, stream);
}

int64_t qs_partition_f64(double *d_keys, int64_t n, double pivot, qs_stream_t stream)
{
    // Under IEEE '<' no key is below a NaN pivot, but no key is at-or-above it either.
    if (pivot != pivot) return fail(QS_ERR_INVALID_ARG, "NaN pivot");
    return run<double>(QS_KIND_F64, d_keys, nullptr, n, bits_f64(pivot), 1, stream);
}

int64_t qs_partition_kv(int32_t *d_keys, int32_t *d_vals, int64_t n, int32_t pivot, qs_stream_t stream)
{
    return run<int32_t>(QS_KIND_KV, d_keys, d_vals, n, bits_i32(pivot), 1, stream);
}

int qs_sort_i32(int32_t *d_keys, int64_t n, qs_stream_t stream)
{
    return static_cast<int>(run<int32_t>(QS_KIND_I32, d_keys, nullptr, n, 0, 0, stream));
}

int qs_sort_f64(double *d_keys, int64_t n, qs_stream_t stream)
{
    return static_cast<int>(run<double>(QS_KIND_F64, d_keys, nullptr, n, 0, 0, stream));
}

int qs_sort_kv(int32_t *d_keys, int32_t *d_vals, int64_t n, qs_stream_t stream)
{
    return static_cast<int>(run<int32_t>(QS_KIND_KV, d_keys, d_vals, n, 0, 0, stream));
}

int qs_sort_segmented_i32(int32_t *d_keys, int64_t n, const int64_t *d_offsets, int64_t nseg, qs_stream_t stream)
{
    return static_cast<int>(run<int32_t>(QS_KIND_I32, d_keys, nullptr, n, 0, 0, stream, d_offsets, nseg));
}

int qs_sort_segmented_f64(double *d_keys, int64_t n, const int64_t *d_offsets, int64_t nseg, qs_stream_t stream)
{
    return static_cast<int>(run<double>(QS_KIND_F64, d_keys, nullptr, n, 0, 0, stream, d_offsets, nseg));
}

int qs_sort_segmented_kv(int32_t *d_keys, int32_t *d_vals, int64_t n, const int64_t *d_offsets, int64_t nseg,
                         qs_stream_t stream)
{
    return static_cast<int>(run<int32_t>(QS_KIND_KV, d_keys, d_vals, n, 0, 0, stream, d_offsets, nseg));
}

int qs_sort_learned_i32(int32_t *d_keys, int64_t n, const float *d_params, qs_stream_t stream)
{
    return run_learned<int32_t>(QS_KIND_I32, d_keys, n, kOpSortLearned, d_params, nullptr, 0, nullptr, nullptr, nullptr,
                                stream);
}

int qs_sort_learned_f64(double *d_keys, int64_t n, const float *d_params, qs_stream_t stream)
{
    return run_learned<double>(QS_KIND_F64, d_keys, n, kOpSortLearned, d_params, nullptr, 0, nullptr, nullptr, nullptr,
                               stream);
}

int qs_bucket_i32(int32_t *d_keys, int64_t n, const int32_t *d_splitters, int nsplit, int64_t *d_bucket_off,
                  qs_stream_t stream)
{
    return run_learned<int32_t>(QS_KIND_I32, d_keys, n, kOpBucket, nullptr, d_splitters, nsplit, d_bucket_off, nullptr,
                                nullptr, stream);
}

int qs_bucket_f64(double *d_keys, int64_t n, const double *d_splitters, int nsplit, int64_t *d_bucket_off,
                  qs_stream_t stream)
{
    return run_learned<double>(QS_KIND_F64, d_keys, n, kOpBucket, nullptr, d_splitters, nsplit, d_bucket_off, nullptr,
                               nullptr, stream);
}

int qs_sketch_i32(const int32_t *d_keys, int64_t n, float *d_sketch, double *d_minmax, int32_t *d_sample,
                  qs_stream_t stream)
{
    return run_learned<int32_t>(QS_KIND_I32, const_cast<int32_t *>(d_keys), n, kOpSketch, nullptr, nullptr, 0, nullptr,
                                d_sketch, d_minmax, stream, d_sample);
}

int qs_sketch_f64(const double *d_keys, int64_t n, float *d_sketch, double *d_minmax, double *d_sample,
                  qs_stream_t stream)
{
    return run_learned<double>(QS_KIND_F64, const_cast<double *>(d_keys), n, kOpSketch, nullptr, nullptr, 0, nullptr,
                               d_sketch, d_minmax, stream, d_sample);
}

int qs_mlp_param_count(void) { return mlp_param_count(); }

int qs_mlp_forward(const float *d_params, const float *d_x, int64_t batch, float *d_q, float *d_act, qs_stream_t stream)
{
    t_error.clear();
    if (batch < 0 || batch > (1 << 20) || !d_params || !d_x || !d_q) return fail(QS_ERR_INVALID_ARG, "bad MLP arguments");
    const int rc = mlp_forward(d_params, d_x, batch, d_q, d_act, stream);
    return rc ? cuda_fail(static_cast<cudaError_t>(rc), "MLP forward") : QS_OK;
}

int qs_mlp_backward(const float *d_params, const float *d_x, const float *d_t, const float *d_act, int64_t batch,
                    float *d_work, float *d_grad, float *d_loss, qs_stream_t stream)
{
    t_error.clear();
    if (batch < 0 || batch > (1 << 20) || !d_params || !d_x || !d_t || !d_act || !d_work || !d_grad)
        return fail(QS_ERR_INVALID_ARG, "bad MLP arguments");
    const int rc = mlp_backward(d_params, d_x, d_t, d_act, batch, d_work, d_grad, d_loss, stream);
    return rc ? cuda_fail(static_cast<cudaError_t>(rc), "MLP backward") : QS_OK;
}

int qs_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int64_t step, float lr,
                qs_stream_t stream)
{
    t_error.clear();
    if (step < 1 || !d_params || !d_grad || !d_m || !d_v) return fail(QS_ERR_INVALID_ARG, "bad Adam arguments");
    const int rc = mlp_adam(d_params, d_grad, d_m, d_v, step, lr, stream);
    return rc ? cuda_fail(static_cast<cudaError_t>(rc), "Adam step") : QS_OK;
}

int qs_sort_host_i32(int32_t *h_keys, int64_t n, qs_stream_t stream)
{
    return run_host<int32_t>(QS_KIND_I32, h_keys, nullptr, n, stream);
}

int qs_sort_host_f64(double *h_keys, int64_t n, qs_stream_t stream)
{
    return run_host<double>(QS_KIND_F64, h_keys, nullptr, n, stream);
}

int qs_sort_host_kv(int32_t *h_keys, int32_t *h_vals, int64_t n, qs_stream_t stream)
{
    return run_host<int32_t>(QS_KIND_KV, h_keys, h_vals, n, stream);
}

int qs_reserve(int64_t n, int kind)
{
    t_error.clear();
    if (n < 0 || n > kMaxN) return fail(QS_ERR_INVALID_ARG, "n out of range");
    if (kind < QS_KIND_I32 || kind > QS_KIND_KV) return fail(QS_ERR_INVALID_ARG, "bad kind %d", kind);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(QS_ERR_INVALID_ARG, "device %d out of range", dev);
    Workspace &w = *workspace_for(dev);
    std::lock_guard<std::mutex> guard(w.mu);
    return ws_ensure(w, n, kind);
}

void qs_release(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
    Workspace &w = *workspace_for(dev);
    std::lock_guard<std::mutex> guard(w.mu);
    ws_free(w);
}

int qs_sync_status(qs_stream_t stream)
{
    t_error.clear();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(QS_ERR_INVALID_ARG, "device %d out of range", dev);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Workspace &w = *workspace_for(dev);
    std::lock_guard<std::mutex> guard(w.mu);
    if (w.init && w.done_recorded && (e = cudaEventSynchronize(w.done)) != cudaSuccess)
        return cuda_fail(e, "cudaEventSynchronize");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (!w.init || !w.unreported) return QS_OK;
    stats_from_ctrl(w);
    const int rc = report_status(w, s);
    if (rc && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}

const char *qs_last_error(void) { return t_error.c_str(); }

int qs_version(void) { return 100; }

int qs_get_stats(qs_stats *out)
{
    if (!out) return QS_ERR_INVALID_ARG;
    *out = t_stats;
    return QS_OK;
}

int qs_set_option(int option, int64_t value)
{
    switch (option) {
    case QS_OPT_PROFILE:
        if (value < 0 || value > 2) return QS_ERR_INVALID_ARG;
        g_profile = static_cast<int>(value);
        return QS_OK;
    case QS_OPT_WAIT_LIMIT_NS:
        if (value < 0) return QS_ERR_INVALID_ARG;
        g_wait_limit_ns = value;
        return QS_OK;
    case QS_OPT_TASK_CAP:
        if (value < 0) return QS_ERR_INVALID_ARG;
        g_task_cap = value;
        return QS_OK;
    case QS_OPT_DRIVER_CTAS:
        if (value < 0 || value > (1 << 20)) return QS_ERR_INVALID_ARG;
        g_driver_ctas = value;
        return QS_OK;
    case QS_OPT_DRIVER_ITEMS:
        if (value < 0 || value > 64) return QS_ERR_INVALID_ARG;
        g_driver_items = value;
        return QS_OK;
    case QS_OPT_ORDERED:
        if (value < 0 || value > 1) return QS_ERR_INVALID_ARG;
        g_ordered = static_cast<int>(value);
        return QS_OK;
    case QS_OPT_SYNC:
        if (value < 0 || value > 1) return QS_ERR_INVALID_ARG;
        g_sync = static_cast<int>(value);
        return QS_OK;
    case QS_OPT_BUCKET_LEVELS:
        if (value < 0 || value > 2) return QS_ERR_INVALID_ARG;
        g_bucket_levels = static_cast<int>(value);
        return QS_OK;
    case QS_OPT_LEAF_MAX:
    case QS_OPT_SMALL_MAX:
        if (value < 0 || (value > 0 && (value < 32 || (value & (value - 1))))) return QS_ERR_INVALID_ARG;
        (option == QS_OPT_LEAF_MAX ? g_leaf_max : g_small_max) = value;
        return QS_OK;
    default:
        return QS_ERR_INVALID_ARG;
    }
}

int qs_get_option(int option, int64_t *value)
{
    if (!value) return QS_ERR_INVALID_ARG;
    switch (option) {
    case QS_OPT_PROFILE: *value = g_profile.load(); return QS_OK;
    case QS_OPT_WAIT_LIMIT_NS: *value = g_wait_limit_ns.load(); return QS_OK;
    case QS_OPT_TASK_CAP: *value = g_task_cap.load(); return QS_OK;
    case QS_OPT_DRIVER_CTAS: *value = g_driver_ctas.load(); return QS_OK;
    case QS_OPT_LEAF_MAX: *value = g_leaf_max.load(); return QS_OK;
    case QS_OPT_SMALL_MAX: *value = g_small_max.load(); return QS_OK;
    case QS_OPT_DRIVER_ITEMS: *value = g_driver_items.load(); return QS_OK;
    case QS_OPT_ORDERED: *value = g_ordered.load(); return QS_OK;
    case QS_OPT_SYNC: *value = g_sync.load(); return QS_OK;
    case QS_OPT_BUCKET_LEVELS: *value = g_bucket_levels.load(); return QS_OK;
    default: return QS_ERR_INVALID_ARG;
    }
}

}  // extern "C"
