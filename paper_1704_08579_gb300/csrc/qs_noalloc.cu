// qs_partition_i32_noalloc: the int32 partition for callers that may not
// allocate device memory.
//
// The regular entry points keep a per-device workspace that they grow with
// cudaMalloc (and shrink with cudaFree, which synchronises the whole device).
// Some callers cannot allow that: code that runs under a fixed device-memory
// budget handed out by its own allocator, code that must never trigger the
// implicit device-wide synchronisation of cudaFree, and code that has to keep
// the allocation count of the process constant.  This entry point needs no
// allocation at all: its scratch memory is one file-scope __device__ array of
// fixed size, sized for at most QS_NOALLOC_MAX_N keys.  Every GPU that loads
// the library holds that array until the process exits.
//
// The kernels are the same as qs_partition_i32's (setup + persistent
// partition kernel), launched on the same ticket/look-back machinery; only the
// place the scratch lives differs.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/qs.h"
#include "qs_internal.h"

namespace qs {
namespace {

constexpr int64_t kMaxN = QS_NOALLOC_MAX_N;
constexpr int64_t kMaxTiles = kMaxN / 1024 + 16;  // every partition tile holds >= 1024 keys
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffKeys = 0;
constexpr size_t kOffPool = align_up(kOffKeys + kMaxN * sizeof(int32_t));
constexpr size_t kOffOwner = align_up(kOffPool + kMaxTiles * sizeof(unsigned long long));
constexpr size_t kOffTask = align_up(kOffOwner + kMaxTiles * sizeof(int32_t));
constexpr size_t kOffLeaf = align_up(kOffTask + sizeof(Task));
constexpr size_t kOffCtrl = align_up(kOffLeaf + sizeof(Leaf));
constexpr size_t kBytes = align_up(kOffCtrl + sizeof(Ctrl));

// The scratch.  In host code this name is only a stand-in for the device
// array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch
    int grid = 0;
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_mu;

// Errors are reported through the return value only (a negative qs_status).
int64_t fail(int64_t code, const char *) { return code; }

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" int64_t qs_partition_i32_noalloc(int32_t *d_keys, int64_t n, int32_t pivot, qs_stream_t stream)
{
    if (n < 0 || n > kMaxN) return fail(QS_ERR_INVALID_ARG, "n out of range [0, QS_NOALLOC_MAX_N]");
    if (n == 0) return 0;
    if (!d_keys) return fail(QS_ERR_INVALID_ARG, "null key pointer");
    if (reinterpret_cast<uintptr_t>(d_keys) % 4) return fail(QS_ERR_ALIGN, "keys not aligned to 4 bytes");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(QS_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return fail(QS_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> guard(g_mu);  // calls share the one scratch array
    DeviceSetup &su = g_setup[dev];
    if (!su.ready) {
        // Once per device, with that device current: the device address of the
        // scratch array and the persistent grid size.
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess)
            return fail(QS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        int sms = 0, bps = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            occupancy_i32(2, &bps) != cudaSuccess || bps < 1)  // the partitions' (narrow) tile
            return fail(QS_ERR_CUDA, "device query failed");
        su.base = static_cast<unsigned char *>(p);
        su.grid = sms * bps;
        su.ready = true;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // The look-back words, ticket owners and the control block (with its
    // status words) start at zero: the previous call may have failed.
    if (cudaMemsetAsync(su.base + kOffPool, 0, kBytes - kOffPool, s) != cudaSuccess)
        return fail(QS_ERR_CUDA, "cudaMemsetAsync failed");

    const KernelLimits lim = limits_i32();
    Args<int32_t, int32_t> a;
    std::memset(&a, 0, sizeof(a));
    a.keys[0] = d_keys;
    a.keys[1] = reinterpret_cast<int32_t *>(su.base + kOffKeys);
    a.key_phase[0] = static_cast<int>((reinterpret_cast<uintptr_t>(d_keys) / 4) % 4);
    a.key_phase[1] = 0;
    a.val_vec[0] = a.val_vec[1] = 1;
    a.n = n;
    a.tasks = reinterpret_cast<Task *>(su.base + kOffTask);
    a.owner = reinterpret_cast<int32_t *>(su.base + kOffOwner);
    a.pool = reinterpret_cast<unsigned long long *>(su.base + kOffPool);
    a.leaves = reinterpret_cast<Leaf *>(su.base + kOffLeaf);
    a.ctrl = reinterpret_cast<Ctrl *>(su.base + kOffCtrl);
    a.task_cap = 1;
    a.pool_cap = kMaxTiles;
    a.leaf_cap = 1;
    a.leaf_max = lim.leaf_max;
    a.small_max = lim.small_max;
    a.wait_limit_ns = option_wait_limit_ns();  // QS_OPT_WAIT_LIMIT_NS, as for qs_partition_i32
    a.pivot_bits = static_cast<uint64_t>(static_cast<int64_t>(pivot));
    a.partition_only = 1;
    a.ordered = 1;
    a.profile = 0;
    a.okeys = a.keys[0];
    a.ovals = a.vals[0];
    LaunchCfg cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.stream = s;
    cfg.grid_driver = su.grid;
    cfg.grid_leaf = su.grid;
    cfg.items = lim.items_default_part;  // the tile qs_partition_i32 uses
    cfg.profile = 0;
    if (launch_i32(a, cfg) != cudaSuccess) return fail(QS_ERR_CUDA, "kernel launch failed");
    Ctrl h;  // pageable host copy of the control block: no host allocation either
    if (cudaMemcpyAsync(&h, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(QS_ERR_CUDA, "reading the result failed");
    if (h.status != 0) return fail(h.status, "device-side failure (see qs_status)");
    // The lower side was written in place; the upper side, [split, n), comes back from scratch.
    const int64_t lt = static_cast<int64_t>(h.lt_result);
    if (lt < 0 || lt > n) return fail(QS_ERR_INTERNAL, "split beyond the array");
    if (lt < n && (cudaMemcpyAsync(d_keys + lt, a.keys[1] + lt, static_cast<size_t>(n - lt) * 4, cudaMemcpyDeviceToDevice,
                                   s) != cudaSuccess ||
                   cudaStreamSynchronize(s) != cudaSuccess))
        return fail(QS_ERR_CUDA, "copy-back failed");
    return lt;
}
