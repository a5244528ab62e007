// Internal declarations shared by the CUDA translation units of libqs.so.
//
// Device-resident state of one sort (all in the per-device workspace):
//   Task   -- one device-wide partition of a range [off, off+len) of buffer
//             `src` (0 = caller's array, 1 = scratch) around `pivot`; split
//             into tiles that any CTA of the persistent kernel may claim.
//   pool   -- look-back words, one per tile of every task (Merrill & Garland
//             single-pass scan with decoupled look-back): 2 flag bits
//             (aggregate available / inclusive prefix available) + 62-bit
//             count of keys sent to the lower side.  A task's tiles own a
//             contiguous range of words, reserved when the task is created;
//             the word index doubles as the tile's global ticket.
//   owner  -- for every ticket, the id (+1) of the task it belongs to
//             (0 = not yet published).  CTAs claim tickets in increasing
//             order with one atomic, so every wait (look-back, task
//             completion) points to a lower ticket and cannot form a cycle.
//   leaves -- parts left for the Bitonic kernel.  "Large" entries fill the
//             array from the front (one CTA each), "small" ones from the back
//             (one warp each).
//   Ctrl   -- queue cursors, allocation cursors, pending-task count, status
//             word and statistics.
#pragma once

#include <cstddef>
#include <cstdint>

namespace qs {

constexpr int kThreads = 256;            // threads per CTA in every kernel
constexpr int kWarps = kThreads / 32;
constexpr int kDThreads = 256;           // default threads per CTA of the persistent partition kernel (Traits::DT)
constexpr int kLThreads = 1024;          // threads per CTA of the leaf kernel (one CTA per SM)
constexpr int kDWarps = kDThreads / 32;

constexpr uint64_t kFlagAggregate = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kCountMask = (1ull << 62) - 1;

constexpr int kMaxDepth = 250;           // deeper recursion => QS_ERR_INTERNAL
constexpr int64_t kCopyChunk = 1 << 15;  // finished equal-key runs are copied in chunks

enum TaskMode : int32_t { kModeLess = 0, kModeLessEqual = 1 };

struct alignas(16) Task {
    int64_t off;        // first element of the range
    int64_t len;        // elements in the range
    int64_t w0;         // first element of tile 0 (16-byte aligned address, <= off)
    int64_t pool;       // index of tile 0's look-back word
    uint64_t pivot;     // key bits (int32 sign-extended, or double bits)
    int32_t ntiles;
    int32_t src;        // buffer holding the range: 0 caller, 1 scratch
    int32_t mode;       // TaskMode
    int32_t depth;
    unsigned long long next_tile;   // tile claim counter
    unsigned long long tiles_done;  // completion counter
    unsigned long long eq;          // keys equal to the pivot
    unsigned long long lt_total;    // keys sent to the lower side (ordered: written by the last tile;
                                    // unordered: the lower side's placement counter)
    unsigned long long hi_total;    // unordered placement: keys sent to the upper side so far
};

struct alignas(16) Leaf {
    int64_t off;
    int32_t len;
    int32_t flags;  // bit 0: range lives in scratch; bit 1: finished (copy only)
};
constexpr int kLeafScratch = 1;
constexpr int kLeafFinal = 2;

constexpr int kProfSlots = 40;  // driver profiling slots (qs_stats.driver_cycles)

struct alignas(128) Ctrl {
    unsigned long long ticket_head;  // next ticket to hand out
    unsigned long long n_tasks, pool_cursor;
    long long pending;  // device-wide partition tasks created and not finished
    unsigned long long n_large, n_small;
    unsigned long long claim_large, claim_small;
    int status, info;
    int sticky, sticky_info;  // first error of an earlier call not yet reported to the host
    // statistics
    unsigned long long part_tasks, part_keys, leaf_parts, leaf_keys, copy_keys, max_depth;
    unsigned long long mid_parts, mid_keys;  // parts split once by the leaf kernel, their keys
    unsigned long long lt_result;  // split index of a partition-only call
    unsigned long long exited;     // CTAs of the persistent kernel that left cleanly
    unsigned long long cycles[kProfSlots];  // per-phase SM cycles and counters (profiling on)
};

// Arguments of the device kernels (passed by value).
template <class K, class V>
struct Args {
    K *keys[2];   // [0] caller array, [1] scratch
    V *vals[2];
    int key_phase[2];  // (address / sizeof(K)) % (16 / sizeof(K)) of each key buffer
    int val_vec[2];    // value buffer shares the key buffer's 16-byte phase
    int64_t n;
    Task *tasks;
    int32_t *owner;  // pool_cap entries
    unsigned long long *pool;
    Leaf *leaves;
    Ctrl *ctrl;
    int64_t task_cap, pool_cap, leaf_cap;  // owner and pool hold pool_cap entries
    int64_t leaf_max;   // parts up to this size go to the leaf kernel
    int64_t small_max;  // parts up to this size are sorted by one warp
    uint64_t wait_limit_ns;
    uint64_t pivot_bits;  // partition-only: the caller's pivot
    int partition_only;
    int ordered;  // 1: tiles placed in input order (look-back); 0: each tile claims its ranges with atomics
    int profile;  // accumulate per-phase cycle counts into ctrl->cycles
    const int64_t *seg_off;  // segmented sort: nseg + 1 offsets into keys (nullptr otherwise)
    int64_t nseg;
    int seg_src;  // buffer holding the segments: 0 caller, 1 scratch
    // Where the leaf kernel writes the sorted result: keys[0] / vals[0], or a
    // separate array (a mapped pinned host buffer of the host-buffer sort),
    // in which case every finished range is copied there, also those that
    // are finished in place in keys[0].
    K *okeys;
    V *ovals;
    int out_separate;
};

// Launch description computed by the host and consumed by the per-kind launchers.
struct LaunchCfg {
    void *stream;
    int grid_driver;
    int grid_leaf;
    int items;  // keys per thread of a partition tile: the narrow variant's, or any other value for the wide one
    int profile;
    void *ev[6];  // cudaEvent_t when profiling
};

// Learned-splitter / bucket pass state (one per workspace; device memory).
constexpr int kLearnedBuckets = 256;
constexpr int kLearnedSketch = 1024;
constexpr int kMaxBucketCtas = 2048;
// Second bucket level: every first-level bucket split 256 ways again, by its
// own sampled splitters; its passes give each CTA one chunk of one bucket.
constexpr int kLearnedBuckets2 = kLearnedBuckets * kLearnedBuckets;
constexpr int64_t kBucket2Chunk = 1 << 16;
struct alignas(128) LearnedState {
    double minmax[2];
    int64_t bucket_off[kLearnedBuckets + 1];  // bucket starts + total (nsplit + 2 used)
    unsigned long long bucket_max;
    unsigned long long bucket_over;  // buckets above the bound
    unsigned long long bucket_dev;   // sum over buckets of |size * nbuckets - n|
    int status;
    int nsplit;
};
struct LearnedPtrs {
    LearnedState *st;
    float *sketch;     // kLearnedSketch floats
    void *sample;      // kLearnedSketch sort-space keys (8 bytes each)
    void *splitters;   // 255 sort-space keys (8 bytes each)
    int64_t *cnt;      // kLearnedBuckets x kMaxBucketCtas
    float *act;        // one sample's MLP activations
    // Second level (sorts with two bucket levels):
    void *spl2;        // kLearnedBuckets x 256 sort-space keys: each bucket's 255 sorted sub-splitters
    int64_t *off2;     // kLearnedBuckets2 + 1 starts of the sub-buckets (the final sort's segments)
    int64_t *cbase;    // kLearnedBuckets + 1: first second-level chunk of each bucket, then the total
    int64_t *cnt2;     // chunks x 256 sub-bucket counts, then cursors
};
enum LearnedOp { kOpSketch = 0, kOpBucket = 1, kOpSortLearned = 2 };
struct LearnedCall {
    LearnedPtrs p;
    int op;
    const float *params;     // MLP parameters (nullptr = sampled splitters)
    const void *user_spl;    // kOpBucket: caller's splitters (raw keys)
    int nsplit;              // kOpBucket: number of caller's splitters (<= 255)
    int ctas;                // CTAs of the bucket kernels
    int levels;              // kOpSortLearned: 1 or 2 bucket levels
    int ctas2;               // CTAs of the second-level passes (an upper bound on the chunks)
    int64_t bound;           // bucket size counted as "over"
    float *sketch_out;       // kOpSketch outputs (device)
    double *minmax_out;
    void *sample_out;        // kOpSketch: sorted sample keys (device, optional)
};

struct KernelLimits {
    int64_t leaf_max, small_max, tile;  // tile: the smaller of the two partition tile variants
    // leaf_max: the largest part the leaf kernel takes (a part above
    // leaf_default is split once by the leaf kernel itself); leaf_default:
    // the threshold used when QS_OPT_LEAF_MAX is 0 (what one CTA's shared
    // memory sorts)
    int64_t leaf_default;
    size_t driver_smem, leaf_smem;
    int items_wide, items_narrow;       // keys per thread of the two partition tile variants
    int items_xwide;                    // keys per thread of the register-tile variant (0: none)
    int items_default;                  // the variant a sort uses when QS_OPT_DRIVER_ITEMS is 0
    int items_default_part;             // the variant a partition-only call uses then
};

// Per-kind entry points implemented in qs_kind_{i32,f64,kv}.cu.  They enqueue
// setup + persistent partition kernel + leaf kernel (sort) or setup +
// persistent kernel (partition only) on cfg.stream and return a cudaError_t.
// With a.seg_off set they sort every segment [seg_off[i], seg_off[i+1]).
int launch_i32(const Args<int32_t, int32_t> &a, LaunchCfg &cfg);
int launch_f64(const Args<double, int32_t> &a, LaunchCfg &cfg);
int launch_kv(const Args<int32_t, int32_t> &a, LaunchCfg &cfg);
// Learned / bucket / sketch operations (i32 and f64 keys).
int learned_i32(const Args<int32_t, int32_t> &a, const LearnedCall &lc, LaunchCfg &cfg);
int learned_f64(const Args<double, int32_t> &a, const LearnedCall &lc, LaunchCfg &cfg);
// MLP kernels (kind-independent).
int mlp_param_count();
int mlp_forward(const float *P, const float *X, int64_t batch, float *Q, float *ACT, void *stream);
int mlp_backward(const float *P, const float *X, const float *T, const float *ACT, int64_t batch, float *WORK,
                 float *G, float *loss, void *stream);
int mlp_adam(float *P, const float *G, float *M, float *V, int64_t step, float lr, void *stream);
// Current QS_OPT_WAIT_LIMIT_NS (shared by every entry point).
uint64_t option_wait_limit_ns();
KernelLimits limits_i32();
KernelLimits limits_f64();
KernelLimits limits_kv();
// Resident CTAs per SM of the persistent kernel (which = 0 wide tile, 2
// narrow tile, 3 register tile) or the leaf kernel (which = 1) of each kind.
int occupancy_i32(int which, int *blocks_per_sm);
int occupancy_f64(int which, int *blocks_per_sm);
int occupancy_kv(int which, int *blocks_per_sm);

}  // namespace qs
