/*
 * qs.h -- C-ABI of the GB300 (sm_103a) hybrid Quicksort library (libqs.so).
 *
 * The operations are those of Bramas, "A Novel Hybrid Quicksort Algorithm
 * Vectorized using AVX-512 on Intel Skylake" (arXiv 1704.08579):
 *   - partition an array around a pivot          (Section III-B, Algorithm 2)
 *   - sort an array in place: partition until the parts are small, then sort
 *     the parts with a branch-free Bitonic network (Sections III-A and III-C,
 *     Algorithm 3; small-array sort Section III-A, Algorithms 1 and 2)
 *   - the same for key/value pairs held in two separate arrays (Section III-D)
 * for three element kinds: int32 keys ("i32"), IEEE double keys ("f64"), and
 * int32 keys carrying int32 values ("kv").
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are CUDA device pointers on the current device.  The
 *     caller owns them; the library never frees or keeps them after the call.
 *     Keys must be aligned to their element size (4 or 8 bytes), values to 4.
 *   - n is an element count, 0 <= n <= 2^38.  n == 0 (and n == 1 for sorts)
 *     succeeds without touching memory.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     issued on it.  qs_sort_* and qs_sort_segmented_* are ASYNCHRONOUS: they
 *     return QS_OK once the work is enqueued (Algorithm 3's simd_QS is a plain
 *     call with no result to wait for), and a device-side failure is reported
 *     later, by qs_sync_status() or by the next call on the device.  Every
 *     other entry point returns only after its work has finished (a partition
 *     returns a split index, the host, learned and bucket forms read results
 *     back).  QS_OPT_SYNC = 1, or profiling, makes the sorts synchronous too.
 *   - The library owns one workspace per device (scratch arrays of n keys and
 *     n values, a task queue, look-back words); it grows on demand or by
 *     qs_reserve(), and is guarded by a mutex, so concurrent host calls on one
 *     device are serialised.  Calls are also ordered on the GPU: each waits
 *     (cudaStreamWaitEvent) for the previous call's last operation, whatever
 *     stream that was issued on, so asynchronous calls on different streams
 *     never overlap on the shared buffers.  A call that has to grow the
 *     workspace (cudaMalloc/cudaFree) synchronises the device; qs_reserve()
 *     beforehand avoids that.
 *   - f64 keys must contain no NaN and no -0.0 (not checked).
 *   - Errors: a negative qs_status; qs_last_error() then describes it.  A
 *     device-side failure (a bounded wait that ran out, a capacity overflow)
 *     leaves the array contents unspecified but a permutation is NOT
 *     guaranteed; the library stays usable.  A failure of an asynchronous
 *     sort is kept in a device status word until it is reported once: by
 *     qs_sync_status(), by a synchronous call, or by the next call that finds
 *     the failed call finished (that call then returns the error and does no
 *     work of its own); qs_last_error() says "an earlier asynchronous call
 *     failed" when the error is not the returning call's own.  Only the first
 *     failure between two reports is kept.
 */
#ifndef QS_H_
#define QS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qs_stream_t; /* == cudaStream_t */

typedef enum {
    QS_OK = 0,
    QS_ERR_INVALID_ARG = -1, /* bad pointer, negative or too large n, bad kind/option */
    QS_ERR_ALIGN = -2,       /* pointer not aligned to its element size */
    QS_ERR_OOM = -3,         /* workspace allocation failed */
    QS_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    QS_ERR_TIMEOUT = -5,     /* a device-side bounded wait ran out */
    QS_ERR_CAPACITY = -6,    /* task / look-back / leaf capacity exceeded on the device */
    QS_ERR_INTERNAL = -7     /* recursion deeper than the supported limit, or an internal
                                consistency check failed (an index that would have been
                                out of range: nothing was written there) */
} qs_status;

typedef enum { QS_KIND_I32 = 0, QS_KIND_F64 = 1, QS_KIND_KV = 2 } qs_kind;

/*
 * Partition (Section III-B): reorders d_keys[0..n) so that every key strictly
 * below `pivot` comes first and every key at-or-above it comes last, and
 * returns the split index = the number of keys below the pivot (the paper's
 * returned left_w), in [0, n].  The order inside each side is fixed: the lower
 * side keeps input order, the upper side holds its keys in reverse input
 * order.  For kv, d_vals[i] moves with d_keys[i].
 * One pass reads every element once: the lower side is written in place
 * (a tile's lower-side keys only land on positions that this tile or an
 * earlier one has already read), the upper side into the workspace scratch,
 * from where it is copied back into d_keys/d_vals once the split is known
 * (2 * n + 2 * (n - split) element moves in all).  Returns a negative
 * qs_status on error (QS_ERR_INVALID_ARG for a NaN pivot, before any work);
 * after a device-side failure the contents of d_keys/d_vals are unspecified
 * (keys may be duplicated or lost).
 */
int64_t qs_partition_i32(int32_t *d_keys, int64_t n, int32_t pivot, qs_stream_t stream);
int64_t qs_partition_f64(double *d_keys, int64_t n, double pivot, qs_stream_t stream);
int64_t qs_partition_kv(int32_t *d_keys, int32_t *d_vals, int64_t n, int32_t pivot,
                        qs_stream_t stream);

/*
 * Sort in place into non-decreasing key order (Section III-C, Algorithm 3):
 * device-wide partitions around sampled-median pivots, driven by one
 * persistent kernel and a device work queue, until every part holds at most
 * a leaf-sized number of keys; a Bitonic network (Section III-A) then sorts
 * each part into d_keys.  Keys equal to a pivot that can no longer be split
 * are finished as a block.  For kv the values follow their keys; the order of
 * values among equal keys is unspecified (the method is not stable).
 * Asynchronous (see the conventions above): returns QS_OK once enqueued, or a
 * negative qs_status for a bad argument, a failed launch or an earlier
 * asynchronous call's failure.  d_keys (and d_vals) must stay valid until
 * the work has finished.
 */
int qs_sort_i32(int32_t *d_keys, int64_t n, qs_stream_t stream);
int qs_sort_f64(double *d_keys, int64_t n, qs_stream_t stream);
int qs_sort_kv(int32_t *d_keys, int32_t *d_vals, int64_t n, qs_stream_t stream);

/*
 * Batched (segmented) sort: sorts every segment [d_offsets[i], d_offsets[i+1])
 * of d_keys (and d_vals) in place, i = 0 .. nseg-1, independently.  d_offsets
 * is a DEVICE array of nseg+1 int64 offsets with 0 <= d_offsets[i] <=
 * d_offsets[i+1] <= n (checked on the device: a bad table returns
 * QS_ERR_INVALID_ARG and leaves the keys unspecified).  All segments are sorted
 * by one setup pass, one launch of the persistent partition kernel and one
 * launch of the leaf kernel; these are captured once per argument set into a
 * CUDA graph and replayed.  Same method and return convention as qs_sort_*
 * (asynchronous).
 */
int qs_sort_segmented_i32(int32_t *d_keys, int64_t n, const int64_t *d_offsets, int64_t nseg,
                          qs_stream_t stream);
int qs_sort_segmented_f64(double *d_keys, int64_t n, const int64_t *d_offsets, int64_t nseg,
                          qs_stream_t stream);
int qs_sort_segmented_kv(int32_t *d_keys, int32_t *d_vals, int64_t n, const int64_t *d_offsets,
                         int64_t nseg, qs_stream_t stream);

/*
 * Learned splitters (a growth line of the method; the paper has no model).
 * The sort keeps the paper's method inside every bucket; what is learned is a
 * set of 255 splitters that cut the array into 256 buckets first:
 *   1. a sketch: 1024 keys sampled at jittered strides, sorted, min-max scaled
 *      to [0,1] (qs_sketch_*);
 *   2. an FP32 MLP 1024 -> 64 (ReLU) -> 64 (ReLU) -> 256 softplus increments,
 *      whose normalised cumulative sums give 255 monotone positions q in
 *      [0,1] along the sorted sample; splitter j is read at position
 *      q_j * 1023 of the sample's curve -- the sorted sample smoothed by a
 *      centred moving average of 17 keys (the window shrinking at both ends)
 *      -- by linear interpolation between neighbouring curve points (rounded
 *      for int32);
 *   3. a 256-way bucket pass: bucket(k) = number of splitters <= k
 *      (qs_bucket_* runs it alone, with the caller's splitters);
 *   4. the plain method on every bucket (the segmented sort).  A bucket that
 *      comes out larger than 4x its even share is simply split further by the
 *      plain sampled-median pivots: that is the fallback, and qs_stats reports
 *      bucket_max / bucket_over as the measure of the model.
 * With QS_OPT_BUCKET_LEVELS = 2 a second 256-way bucket pass runs inside
 * every bucket first (its 255 splitters sampled from the bucket itself:
 * 1024 keys, every 4th of them sorted), and step 4 sorts the 65,536
 * sub-buckets -- most of them small enough for the leaf kernel alone.
 * Step 4's partition passes use the kind's first compiled tile (int32: the
 * register tile; FP64: the wide prefetched tile), not QS_OPT_DRIVER_ITEMS.
 * The sorted output is the same as qs_sort_*'s (keys bit for bit).
 *
 * d_params: device float array of qs_mlp_param_count() parameters laid out as
 * W1 (64x1024, row-major), b1 (64), W2 (64x64), b2 (64), W3 (256x64), b3
 * (256), all finite (not checked); NULL = sampled splitters (every 4th key of
 * the sorted sketch sample), the same bucket machinery without the model.
 * Whatever finite parameters give, the sorted output is the same: a key's
 * bucket never decreases as the key grows, for any set of splitters.  Arrays
 * below 2^16 keys use the plain method.  Synchronous; returns QS_OK or a
 * negative qs_status.
 */
int qs_sort_learned_i32(int32_t *d_keys, int64_t n, const float *d_params, qs_stream_t stream);
int qs_sort_learned_f64(double *d_keys, int64_t n, const float *d_params, qs_stream_t stream);

/*
 * Bucket pass alone: reorders d_keys[0..n) so that bucket b = the keys with
 * exactly b of the nsplit (1..255, non-decreasing, device array) splitters <=
 * key come before bucket b+1; the order inside a bucket is unspecified.
 * d_bucket_off (device, nsplit + 2 int64) receives the bucket starts and n.
 * Synchronous; returns QS_OK or a negative qs_status.
 */
int qs_bucket_i32(int32_t *d_keys, int64_t n, const int32_t *d_splitters, int nsplit, int64_t *d_bucket_off,
                  qs_stream_t stream);
int qs_bucket_f64(double *d_keys, int64_t n, const double *d_splitters, int nsplit, int64_t *d_bucket_off,
                  qs_stream_t stream);

/*
 * Sketch of n >= 1024 keys: d_sketch (device, 1024 floats) = the sorted sample
 * scaled to [0,1], d_minmax (device, 2 doubles) = its smallest and largest
 * key, d_sample (device, 1024 keys, or NULL) = the sorted sample keys.  This
 * is the MLP's input.  Synchronous.
 */
int qs_sketch_i32(const int32_t *d_keys, int64_t n, float *d_sketch, double *d_minmax, int32_t *d_sample,
                  qs_stream_t stream);
int qs_sketch_f64(const double *d_keys, int64_t n, float *d_sketch, double *d_minmax, double *d_sample,
                  qs_stream_t stream);

/*
 * Training kernels of the splitter MLP (FP32, all device pointers, asynchronous
 * on `stream`; they return after enqueueing).
 *   qs_mlp_param_count  number of parameters (86400).
 *   qs_mlp_forward      d_x: batch x 1024 sketches -> d_q: batch x 255
 *                       quantiles; d_act (batch x 640 floats, or NULL) keeps
 *                       the activations for backward.
 *   qs_mlp_backward     d_t: batch x 255 targets; gradient of the loss
 *                       mean((q - t)^2) over batch x 255 into d_grad
 *                       (param_count floats, overwritten), the loss into
 *                       *d_loss (or NULL); d_work: batch x 384 floats scratch.
 *   qs_mlp_adam         one Adam step (beta 0.9/0.999, eps 1e-8, bias
 *                       corrected; step counts from 1) on d_params with
 *                       moments d_m, d_v.
 */
int qs_mlp_param_count(void);
int qs_mlp_forward(const float *d_params, const float *d_x, int64_t batch, float *d_q, float *d_act,
                   qs_stream_t stream);
int qs_mlp_backward(const float *d_params, const float *d_x, const float *d_t, const float *d_act,
                    int64_t batch, float *d_work, float *d_grad, float *d_loss, qs_stream_t stream);
int qs_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int64_t step, float lr,
                qs_stream_t stream);

/*
 * Host-buffer sorts: h_keys (and h_vals) are HOST pointers (pinned memory is
 * fastest).  The library copies them into a device staging area owned by the
 * workspace and sorts there with the qs_sort_* path, all on `stream`.  If the
 * buffers are pinned memory mapped into the device's address space (what
 * cudaHostAlloc / cudaMallocHost give under unified addressing), the leaf
 * kernel writes each sorted part straight into them, so the return transfer
 * overlaps the leaf sorts; otherwise the result is copied back afterwards.
 * Synchronous: returns once the host buffers hold the result, QS_OK or a
 * negative qs_status.  Host-buffer sorts on one device share its staging
 * area: calls from several host threads run one after another.
 */
int qs_sort_host_i32(int32_t *h_keys, int64_t n, qs_stream_t stream);
int qs_sort_host_f64(double *h_keys, int64_t n, qs_stream_t stream);
int qs_sort_host_kv(int32_t *h_keys, int32_t *h_vals, int64_t n, qs_stream_t stream);

/*
 * qs_partition_i32 for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a service of the library, not part of
 * the method.  The regular entry points grow a per-device workspace with
 * cudaMalloc (and free it with cudaFree, which synchronises the device); a
 * caller working inside a fixed device-memory budget owned by its own
 * allocator, or one that must never cause that implicit synchronisation,
 * cannot let them.  This variant allocates nothing: its scratch is one fixed
 * file-scope device array of 4,208,128 bytes (4.0 MiB) that every GPU loading the library
 * holds until the process exits.
 *   - Same operation, arguments, result order, return value and wait limit
 *     (QS_OPT_WAIT_LIMIT_NS) as qs_partition_i32, for 0 <= n <=
 *     QS_NOALLOC_MAX_N; a larger n returns QS_ERR_INVALID_ARG.  Errors come
 *     back as a negative qs_status only (qs_last_error is not updated).
 *     Synchronous, like qs_partition_i32.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and the grid size; make that first call before
 *     any stream capture.
 *   - All calls share the one array: the library serialises calls made from
 *     host threads, but work that overlaps on the GPU through any other route
 *     would race on it.  The look-back words are cleared at the start of
 *     every call; the rest is overwritten before it is read.
 */
#define QS_NOALLOC_MAX_N (1 << 20)
int64_t qs_partition_i32_noalloc(int32_t *d_keys, int64_t n, int32_t pivot, qs_stream_t stream);

/*
 * Grows the current device's workspace so that calls of `kind` with up to n
 * elements allocate nothing.  Returns QS_OK or a negative qs_status.
 */
int qs_reserve(int64_t n, int kind);

/* Frees the current device's workspace (a later call re-creates it). */
void qs_release(void);

/*
 * Waits until every call issued on this device's workspace, and all work on
 * `stream`, has finished; then returns QS_OK, or the first device-side failure
 * of an asynchronous call that has not been reported yet (which is then
 * cleared).  Afterwards qs_get_stats() holds the device counters of the last
 * call.  This is the synchronisation point of the asynchronous sorts.
 */
int qs_sync_status(qs_stream_t stream);

/* Text of the last error raised on this host thread ("" if none). */
const char *qs_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int qs_version(void);

/*
 * Counters of the last qs_sort_* / qs_partition_* call on this host thread
 * (for an asynchronous sort: once qs_sync_status() has returned).
 * The byte figures let a caller compute the HBM traffic the schedule moves:
 * every element of a device-wide partition is read once and written once,
 * so are leaf-sorted and copied elements.
 */
typedef struct {
    int64_t n;              /* elements in the call */
    int64_t kind;           /* qs_kind */
    int64_t part_tasks;     /* device-wide partition passes run */
    int64_t part_keys;      /* sum of their lengths */
    int64_t leaf_parts;     /* parts sorted by the Bitonic leaf kernel */
    int64_t leaf_keys;      /* sum of their lengths */
    int64_t copy_keys;      /* finished equal-key elements copied back from scratch */
    int64_t max_depth;      /* deepest partition level reached */
    int64_t lookback_words; /* look-back words used */
    int64_t grid_driver;    /* CTAs of the persistent partition kernel */
    int64_t grid_leaf;      /* CTAs of the leaf kernel */
    double ms_driver;       /* device time of the partition kernel (profiling on) */
    double ms_leaf;         /* device time of the leaf kernel (profiling on) */
    double ms_copy;         /* device time of the partition copy-back (profiling on) */
    double ms_total;        /* device time of the whole call (profiling on) */
    /* QS_OPT_PROFILE = 2: SM clock cycles the persistent kernel's CTAs spent, summed
     * over CTAs, in [0] waiting for work, [1] waiting for a tile's keys,
     * [2] comparing and counting, [3] placing the tile (look-back or range
     * claims) and staging, [4] storing,
     * [5] releasing the tile, [6] completing tasks (pivots, children);
     * [7] = tiles processed; [8] cycles inside the look-back proper, or the
     * range claims and staging of unordered placement (warp 0),
     * [9] cycles the middle warps waited for the prefetched tile, [10] look-back
     * windows of 32 words read, [11] re-reads of unpublished words (ordered
     * placement; unordered: [9] the release fence, [10] the release atomic,
     * [11] issuing the ticket claim);
     * [13] claiming and resolving the next ticket and issuing its load
     * (thread 0); [12], [14], [15] placement phase as seen by the counting
     * warps, warp 0 and the last warp; [16] staging (warp 0), [17] staging
     * (last warp), [18] the count phase's compare-and-ballot work (thread 0);
     * leaf kernel: [19] packing parts into thread groups (thread 0), per
     * group [20] loading, [21] the network, [23] storing, and [22] padding
     * slots sorted; [24] resolving the next ticket, [25] issuing its load
     * (thread 0); [26] sampling the children's pivots, [27] allocating them,
     * [28] publishing their tickets (task completion); leaf kernel's
     * mid-range splits (thread 0): [29] cycles in splits, [30] splits,
     * [31] pivot sampling, [32] loading and counting the chunks, [33]
     * waiting at the chunk barrier, [34] scan and placement. */
    int64_t driver_cycles[40];
    int64_t bucket_max;     /* learned / bucket pass: largest bucket */
    int64_t bucket_over;    /* learned / bucket pass: buckets above 4x their even share */
    int64_t bucket_dev;     /* learned / bucket pass: sum over the B buckets of |size * B - n|;
                               bucket_dev / (2 n B) is the imbalance error (total variation
                               distance between the bucket sizes and an even split) */
    int64_t mid_parts;      /* parts the leaf kernel split once itself (larger than one CTA's
                               shared memory holds: 16384 keys for f64 / kv, 32768 for i32) */
    int64_t mid_keys;       /* their keys: each read once more and written once more, in L2 */
} qs_stats;

int qs_get_stats(qs_stats *out);

/*
 * Options (process-wide).  Returns QS_OK or QS_ERR_INVALID_ARG.
 *   QS_OPT_PROFILE       1: record CUDA events around each kernel of a
 *                        call, on the call's stream (fills ms_* in qs_stats);
 *                        2: also count SM cycles per phase inside the
 *                        kernels (fills driver_cycles; the counting itself
 *                        slows the kernels a little); 0: off.
 *   QS_OPT_WAIT_LIMIT_NS limit of every device-side wait (default 2e9 ns);
 *                        a wait that runs out ends the kernel with
 *                        QS_ERR_TIMEOUT instead of hanging.
 *   QS_OPT_TASK_CAP      if > 0, caps the device task table (to exercise
 *                        QS_ERR_CAPACITY); 0 = size from n.
 *   QS_OPT_DRIVER_CTAS   if > 0, number of CTAs of the persistent kernels;
 *                        0 = all resident CTAs.
 *   QS_OPT_LEAF_MAX      parts of at most this many keys (a power of two,
 *                        >= 32) go to the leaf kernel; 0 = what one CTA's
 *                        shared memory sorts (16384 f64/kv, 32768 i32).
 *                        Up to twice that is accepted (larger values are
 *                        clamped): a part above the shared-memory size is
 *                        then split once around a sampled pivot by the leaf
 *                        kernel's CTA itself, through L2, instead of by one
 *                        more device-wide partition pass (measured slower on
 *                        GB300 for uniform keys, hence not the default).
 *   QS_OPT_SMALL_MAX     parts of at most this many keys (power of two, >= 32)
 *                        are sorted by one warp; 0 = the compiled maximum 512.
 *   QS_OPT_DRIVER_ITEMS  keys per thread of a partition tile: f64 and kv have
 *                        a wide and a narrow prefetched variant (16 / 8;
 *                        the next tile brought into shared memory by a TMA
 *                        copy) and a register tile of 20 keys per thread
 *                        (128-thread CTAs, 20 KB, loaded straight into
 *                        registers, no prefetch buffer, 6 CTAs per SM);
 *                        i32 has a register tile of
 *                        32 keys per thread (32 KB, 4 CTAs per SM) and a
 *                        narrow prefetched variant of 16; the narrow or
 *                        register-tile value selects that variant, any other
 *                        non-zero value the wide one (i32: the register
 *                        tile), 0 the kind's default: for sorts the register
 *                        tile; for partitions i32 narrow, f64 and kv wide.
 *   QS_OPT_ORDERED       0 (default): inside a sort, each partition tile
 *                        claims its lower- and upper-side output ranges with
 *                        one atomic add each on its task's two counters, so
 *                        tiles land in claim order; 1: tiles are placed in
 *                        input order by the decoupled look-back, as in
 *                        qs_partition_* (which always does so).  The sorted
 *                        keys are the same either way; with key/value pairs
 *                        the order of the values of equal keys may differ.
 *   QS_OPT_SYNC          1: qs_sort_* and qs_sort_segmented_* return only
 *                        after their work has finished, with its status;
 *                        0 (default): they are asynchronous.
 *   QS_OPT_BUCKET_LEVELS qs_sort_learned_*: 1 = one 256-way bucket pass, the
 *                        plain method inside each bucket; 2 = a second
 *                        256-way pass inside every bucket, then the plain
 *                        method inside each of the 65,536 sub-buckets;
 *                        0 = the default (2).
 * The tuning options are what the autotuner (paper_1704_08579_gb300.autotune)
 * searches.
 */
enum {
    QS_OPT_PROFILE = 1,
    QS_OPT_WAIT_LIMIT_NS = 2,
    QS_OPT_TASK_CAP = 3,
    QS_OPT_DRIVER_CTAS = 4,
    QS_OPT_LEAF_MAX = 5,
    QS_OPT_SMALL_MAX = 6,
    QS_OPT_DRIVER_ITEMS = 7,
    QS_OPT_ORDERED = 8,
    QS_OPT_SYNC = 9,
    QS_OPT_BUCKET_LEVELS = 10
};
int qs_set_option(int option, int64_t value);
/* Current value of an option (as set, 0 = the default) into *value; returns
 * QS_OK, or QS_ERR_INVALID_ARG for an unknown option or a NULL pointer. */
int qs_get_option(int option, int64_t *value);

#ifdef __cplusplus
}
#endif

#endif /* QS_H_ */
