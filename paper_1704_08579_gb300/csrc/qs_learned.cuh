// Learned-splitter form of the sort (growth line of the method):
//   sketch_kernel    1024 keys sampled at jittered strides, sorted with the
//                    Bitonic group network, min-max scaled to [0,1] (FP32);
//   splitter_kernel  255 splitters: the MLP's monotone quantile positions
//                    along the sorted sample's moving-average curve, mapped
//                    back to keys by interpolating between curve points
//                    (learned), or every 4th sorted sample key (sampled);
//   bucket_hist / bucket_scan / bucket_scatter
//                    256-way partition by the splitters: bucket(k) = number
//                    of splitters <= k (binary search in shared memory);
//                    per-CTA histograms, one scan, then a scatter that stages
//                    every tile in bucket order so each bucket's keys leave
//                    the CTA as one contiguous run.
// The buckets then go to the segmented sort (plain method).  A bucket that is
// larger than the bound is simply split further by the plain sampled-median
// pivots: that is the fallback.
#pragma once

#include "qs_bitonic.cuh"
#include "qs_common.cuh"
#include "qs_mlp.cuh"

namespace qs {

constexpr int kSketchN = kLearnedSketch;
constexpr int kBuckets = kLearnedBuckets;

template <class K>
struct LearnedBufs {
    LearnedState *st;
    float *sketch;                         // 1024
    typename KeyOps<K>::S *sample;         // 1024 sorted sample keys (sort space)
    typename KeyOps<K>::S *splitters;      // 255 (sort space)
    int64_t *cnt;                          // kBuckets x ctas (bucket-major)
    float *act;                            // MLP activations of one sample
    typename KeyOps<K>::S *spl2;           // second level: 256 x 256 (each bucket's 255 sorted splitters)
    int64_t *off2;                         // kLearnedBuckets2 + 1 sub-bucket starts
    int64_t *cbase;                        // kBuckets + 1 first chunk of each bucket, then the total
    int64_t *cnt2;                         // per bucket j: 256 x chunks_j counts (sub-bucket-major)
};

template <class K>
LearnedBufs<K> bufs_of(const LearnedPtrs &p)
{
    LearnedBufs<K> b;
    b.st = p.st;
    b.sketch = p.sketch;
    b.sample = static_cast<typename KeyOps<K>::S *>(p.sample);
    b.splitters = static_cast<typename KeyOps<K>::S *>(p.splitters);
    b.cnt = p.cnt;
    b.act = p.act;
    b.spl2 = static_cast<typename KeyOps<K>::S *>(p.spl2);
    b.off2 = p.off2;
    b.cbase = p.cbase;
    b.cnt2 = p.cnt2;
    return b;
}

// The caller's splitters (raw keys) in sort space.
template <class K>
__global__ void splitters_from_keys_kernel(const K *__restrict__ spl, int nsplit, LearnedBufs<K> lb)
{
    const int t = threadIdx.x;
    if (t < nsplit) lb.splitters[t] = KeyOps<K>::to_s(spl[t]);
    if (t == 0) {
        lb.st->nsplit = nsplit;
        lb.st->status = 0;
    }
}

// Sketch: one CTA of 256 threads.
template <class K>
__global__ void __launch_bounds__(256) sketch_kernel(const K *__restrict__ keys, int64_t n, LearnedBufs<K> lb,
                                                     float *__restrict__ sketch_out, double *__restrict__ minmax_out,
                                                     K *__restrict__ sample_out)
{
    using Ops = KeyOps<K>;
    using S = typename Ops::S;
    constexpr int E = sizeof(S) == 8 ? 16 : 32, LE = sizeof(S) == 8 ? 4 : 5;
    constexpr int NG = kSketchN / E;  // threads of the sorting group
    __shared__ S sm[kSketchN + kSketchN / 16];
    const int t = threadIdx.x;
    const int64_t stride = n / kSketchN;
    for (int i = t; i < kSketchN; i += 256) {
        const uint64_t h = mix64(0xC0FFEEull * 64 + i);
        const int64_t pos = (static_cast<int64_t>(i) * n) / kSketchN +
                            static_cast<int64_t>(h % static_cast<uint64_t>(stride > 0 ? stride : 1));
        sm[padk<S>(i)] = Ops::to_s(keys[pos < n ? pos : n - 1]);
    }
    __syncthreads();
    if (t < NG) {
        S k[E];
        lay_load<E, LE, S>(k, sm, t, 0);
        group_bitonic_sort<E, LE, 10, S>(k, sm, t, 1, NG);
        group_sync(1, NG);
        lay_store<E, LE, S>(k, sm, t, 0);
    }
    __syncthreads();
    const double lo = static_cast<double>(Ops::from_s(sm[padk<S>(0)]));
    const double hi = static_cast<double>(Ops::from_s(sm[padk<S>(kSketchN - 1)]));
    const double span = hi - lo;
    for (int i = t; i < kSketchN; i += 256) {
        const S s = sm[padk<S>(i)];
        lb.sample[i] = s;
        const double v = static_cast<double>(Ops::from_s(s));
        const float x = span > 0 ? static_cast<float>((v - lo) / span) : 0.f;
        lb.sketch[i] = x;
        if (sketch_out) sketch_out[i] = x;
        if (sample_out) sample_out[i] = Ops::from_s(s);
    }
    if (t == 0) {
        lb.st->status = 0;
        lb.st->minmax[0] = lo;
        lb.st->minmax[1] = hi;
        if (minmax_out) {
            minmax_out[0] = lo;
            minmax_out[1] = hi;
        }
    }
}

// The curve the model's positions are read on: the sorted sample smoothed by
// a centred moving average over kCurveW keys (the window shrinks
// symmetrically at both ends, so the first and last keys stay the sample's
// minimum and maximum).  A moving average of a sorted sequence is
// non-decreasing.  The sample's own bucket noise (about four sample keys per
// bucket) is high-frequency; the network's output, a 64-wide bottleneck,
// can only move the splitters smoothly, so it works on a curve from which
// that noise is already averaged out.
constexpr int kCurveHalf = 8, kCurveW = 2 * kCurveHalf + 1;

template <class K>
__device__ __forceinline__ void sample_curve(const typename KeyOps<K>::S *sample, double *curve)
{
    using Ops = KeyOps<K>;
    for (int i = threadIdx.x; i < kSketchN; i += blockDim.x) {
        const int lo = i - kCurveHalf < 0 ? 0 : i - kCurveHalf;
        const int hi = i + kCurveHalf > kSketchN - 1 ? kSketchN - 1 : i + kCurveHalf;
        const int h = (i - lo) < (hi - i) ? (i - lo) : (hi - i);
        double s = 0;
        for (int k = i - h; k <= i + h; ++k) s += static_cast<double>(Ops::from_s(sample[k]));
        curve[i] = s / (2 * h + 1);
    }
}

// Splitter from quantile position q in [0,1] along the curve: linear
// interpolation between neighbouring curve points, rounded to the key type.
template <class K>
__device__ __forceinline__ K key_at_position(const double *curve, float q)
{
    const double p = static_cast<double>(q < 0.f ? 0.f : (q > 1.f ? 1.f : q)) * (kSketchN - 1);
    const int i = static_cast<int>(p);
    if (i >= kSketchN - 1) return static_cast<K>(curve[kSketchN - 1]);
    const double a = curve[i], b = curve[i + 1];
    double v = a + (p - i) * (b - a);
    v = v < a ? a : (v > b ? b : v);
    if constexpr (sizeof(K) == 4) {
        const double r = rint(v);  // between two int32 means: stays in range
        return static_cast<K>(static_cast<long long>(r));
    } else {
        return v;
    }
}

// Splitters: learned (params != nullptr) or sampled.  One CTA of 256 threads.
// The model's q_j is a position along the smoothed sample curve; the sampled
// form takes every 4th sample key.
template <class K>
__global__ void __launch_bounds__(256) splitter_kernel(const float *__restrict__ params, LearnedBufs<K> lb)
{
    using Ops = KeyOps<K>;
    using S = typename Ops::S;
    __shared__ mlp::Smem sm;
    __shared__ S spl[mlp::kSplit];
    __shared__ double curve[kSketchN];
    const int t = threadIdx.x;
    if (params) {
        for (int i = t; i < kSketchN; i += 256) sm.x[i] = lb.sketch[i];
        sample_curve<K>(lb.sample, curve);
        __syncthreads();
        mlp::forward_cta(params, sm);
        if (t < mlp::kSplit) spl[t] = Ops::to_s(key_at_position<K>(curve, sm.c[t] / sm.c[mlp::kOut - 1]));
    } else if (t < mlp::kSplit) {
        spl[t] = lb.sample[4 * (t + 1)];
    }
    __syncthreads();
    if (t == 0) {  // non-decreasing (positions are monotone; this only guards rounding)
        for (int i = 1; i < mlp::kSplit; ++i)
            if (spl[i] < spl[i - 1]) spl[i] = spl[i - 1];
        lb.st->nsplit = mlp::kSplit;
    }
    __syncthreads();
    if (t < mlp::kSplit) lb.splitters[t] = spl[t];
}

// Bucket of sort-space key s: the number of splitters <= s.  The 255
// (padded) splitters are kept in shared memory as a complete binary search
// tree in breadth-first order (tree[1..255]; node i at depth k holds the
// sorted splitter (2p+1)*2^(8-k)-1, p = i - 2^(k-1)), so the search is
// branch-free and the nodes a warp reads at depth k lie in 2^(k-1)
// consecutive words: no bank conflicts down to depth 6, at most 4-way below.
// (A search over the sorted array reads addresses 2^(9-k) words apart, up to
// 8-way conflicted.)  The leaf reached, minus 256, is the count.
template <class S>
__device__ __forceinline__ int bucket_of(const S *tree, S s)
{
    int i = 1;
#pragma unroll
    for (int d = 0; d < 8; ++d) i = 2 * i + (s < tree[i] ? 0 : 1);
    return i - 256;
}

template <class Tr>
struct BucketSmem {
    typename KeyOps<typename Tr::K>::S spl[256];  // search tree, nodes 1..255
    int hist[kWarps][kBuckets];
};

// Loads `nsplit` sorted splitters into shared memory as the search tree,
// padding the unused slots with the largest key.  Only a key equal to the
// largest key can count a pad; such a key belongs to the last bucket anyway,
// so callers clamp the bucket to nsplit.
template <class K>
__device__ __forceinline__ void load_tree(typename KeyOps<K>::S *tree, const typename KeyOps<K>::S *sorted, int nsplit)
{
    using Ops = KeyOps<K>;
    for (int i = threadIdx.x + 1; i < 256; i += kThreads) {
        const int k = 31 - __clz(i);  // depth - 1
        const int r = (2 * (i - (1 << k)) + 1) * (1 << (7 - k)) - 1;  // sorted index
        tree[i] = r < nsplit ? sorted[r] : Ops::s_largest();
    }
}

// Keys per thread per tile of the bucket pass (16 KB tiles).
template <class K>
constexpr int bucket_e() { return sizeof(K) == 8 ? 8 : 16; }

// Pulls the lines of the chunk's tiles after the current one towards L2 (the
// bucket kernels process their chunk tile by tile; each tile's loads would
// otherwise wait on HBM with nothing else in flight).  One 128-byte line per
// thread and tile, `ahead` tiles of `tile` elements starting at `from`.
template <class T>
__device__ __forceinline__ void prefetch_tiles_l2(const T *p, int64_t from, int64_t hi, int tile, int ahead)
{
    constexpr int kPerLine = 128 / static_cast<int>(sizeof(T));
    for (int t = 0; t < ahead; ++t) {
        const int64_t first = from + static_cast<int64_t>(t) * tile;
        for (int64_t e = first + static_cast<int64_t>(threadIdx.x) * kPerLine; e < first + tile && e < hi;
             e += static_cast<int64_t>(kThreads) * kPerLine)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p + e));
    }
}

// Histogram of keys [lo, hi) over the tree in sm.spl (loaded by the caller,
// followed by a barrier): the count of bucket b goes to cnt[b * stride].
template <class Tr>
__device__ __forceinline__ void hist_range(const typename Tr::K *__restrict__ keys, int64_t lo, int64_t hi,
                                           BucketSmem<Tr> &sm, int nsplit, int64_t *cnt, int64_t stride)
{
    using Ops = KeyOps<typename Tr::K>;
    constexpr int E = bucket_e<typename Tr::K>(), TILE = kThreads * E;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < kWarps * kBuckets; i += kThreads) (&sm.hist[0][0])[i] = 0;
    __syncthreads();
    for (int64_t base = lo; base < hi; base += TILE) {
        // Keep two tiles ahead in L2 (the first tile also covers itself).
        if (base == lo)
            prefetch_tiles_l2(keys, base, hi, TILE, 3);
        else
            prefetch_tiles_l2(keys, base + 2 * TILE, hi, TILE, 1);
        // E independent loads and searches per thread, then one shared-memory
        // add per key into the warp's own histogram.
        typename Ops::S k[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int64_t i = base + j * kThreads + tid;
            k[j] = i < hi ? Ops::to_s(keys[i]) : Ops::s_largest();
        }
        int bk[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int bb = bucket_of(sm.spl, k[j]);
            bk[j] = bb > nsplit ? nsplit : bb;
        }
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (base + j * kThreads + tid < hi) atomicAdd(&sm.hist[warp][bk[j]], 1);
    }
    __syncthreads();
    for (int bb = tid; bb < kBuckets; bb += kThreads) {
        int sum = 0;
        for (int w = 0; w < kWarps; ++w) sum += sm.hist[w][bb];
        cnt[static_cast<int64_t>(bb) * stride] = sum;
    }
}

// First level: CTA c of g takes keys [c*n/g, (c+1)*n/g).
template <class Tr>
__global__ void __launch_bounds__(kThreads) bucket_hist_kernel(const typename Tr::K *__restrict__ keys, int64_t n,
                                                               LearnedBufs<typename Tr::K> lb, int nsplit)
{
    __shared__ BucketSmem<Tr> sm;
    load_tree<typename Tr::K>(sm.spl, lb.splitters, nsplit);
    const int64_t c = blockIdx.x, g = gridDim.x;
    hist_range<Tr>(keys, c * n / g, (c + 1) * n / g, sm, nsplit, lb.cnt + c, g);
}

// Exclusive scan over (bucket, cta) counts in bucket-major order, by one CTA
// of 1024 threads: every count becomes the first slot of its (bucket, CTA)
// run, base + all counts before it, and starts[b] = bucket b's first slot.
// Warp w owns the rows (buckets) w, w+32, ...; lane l a contiguous chunk of
// ceil(ctas/32) counts of a row.  Row totals are scanned once across the CTA,
// then every count is replaced by its prefix.
__device__ __forceinline__ void scan_rows(int64_t *__restrict__ cnt, int ctas, long long base, int64_t *starts)
{
    __shared__ long long tot[kBuckets];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int m = (ctas + 31) / 32;  // counts per lane
    for (int b = warp; b < kBuckets; b += 32) {
        const int64_t *row = cnt + static_cast<int64_t>(b) * ctas;
        long long s = 0;
        for (int j = lane * m; j < (lane + 1) * m && j < ctas; ++j) s += row[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) tot[b] = s;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 256 row totals, 8 per lane
        long long v[kBuckets / 32], sum = 0;
#pragma unroll
        for (int i = 0; i < kBuckets / 32; ++i) {
            v[i] = tot[lane * (kBuckets / 32) + i];
            sum += v[i];
        }
        long long incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        long long run = base + incl - sum;
#pragma unroll
        for (int i = 0; i < kBuckets / 32; ++i) {
            tot[lane * (kBuckets / 32) + i] = run;
            run += v[i];
        }
    }
    __syncthreads();
    for (int b = warp; b < kBuckets; b += 32) {
        int64_t *row = cnt + static_cast<int64_t>(b) * ctas;
        long long s = 0;
        for (int j = lane * m; j < (lane + 1) * m && j < ctas; ++j) s += row[j];
        long long incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        long long run = tot[b] + incl - s;
        for (int j = lane * m; j < (lane + 1) * m && j < ctas; ++j) {
            const long long v = row[j];
            row[j] = run;
            run += v;
        }
        if (lane == 0) starts[b] = tot[b];
    }
}

// First level: one CTA scans the (bucket, CTA) counts, records the bucket
// starts and the bucket statistics.
static __global__ void __launch_bounds__(1024) bucket_scan_kernel(int64_t *__restrict__ cnt, int ctas, LearnedState *st,
                                                           int nsplit, int64_t n, int64_t bound)
{
    const int t = threadIdx.x;
    scan_rows(cnt, ctas, 0, st->bucket_off);
    if (t == 0) st->bucket_off[nsplit + 1] = n;
    __syncthreads();
    // Bucket statistics, one thread per bucket, reduced over the CTA.
    __shared__ unsigned long long red[3][32];
    unsigned long long sz = 0, over = 0, dev = 0;
    if (t <= nsplit) {
        sz = static_cast<unsigned long long>(st->bucket_off[t + 1] - st->bucket_off[t]);
        over = sz > static_cast<unsigned long long>(bound) ? 1 : 0;
        const long long d = static_cast<long long>(sz) * (nsplit + 1) - n;  // vs the even share n/(nsplit+1)
        dev = static_cast<unsigned long long>(d < 0 ? -d : d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long m = __shfl_xor_sync(0xffffffffu, sz, o);
        sz = m > sz ? m : sz;
        over += __shfl_xor_sync(0xffffffffu, over, o);
        dev += __shfl_xor_sync(0xffffffffu, dev, o);
    }
    if ((t & 31) == 0) {
        red[0][t >> 5] = sz;
        red[1][t >> 5] = over;
        red[2][t >> 5] = dev;
    }
    __syncthreads();
    if (t == 0) {
        unsigned long long mx = 0, ov = 0, dv = 0;
        for (int w = 0; w < 32; ++w) {
            mx = red[0][w] > mx ? red[0][w] : mx;
            ov += red[1][w];
            dv += red[2][w];
        }
        st->bucket_max = mx;
        st->bucket_over = ov;
        st->bucket_dev = dv;
    }
}

static_assert(kThreads == kBuckets, "one thread per bucket in the scatter's per-tile bookkeeping");

template <class Tr>
struct ScatterSmem {
    static constexpr int TILE = kThreads * bucket_e<typename Tr::K>();
    typename KeyOps<typename Tr::K>::S spl[256];  // search tree, nodes 1..255
    typename Tr::K keys[TILE];
    typename Tr::V vals[Tr::KV ? TILE : 1];
    unsigned char bkt[TILE];
    int tcnt[kBuckets];
    int tstart[kBuckets];
    long long cursor[kBuckets];
    int wsum[kWarps];
};

// Scatter of keys [lo, hi) from sk/sv to dk/dv: each tile's keys are ranked
// inside their buckets with one shared atomic per key, staged in bucket
// order, and leave the CTA as one contiguous run per (tile, bucket).  The
// tree is in sm.spl (loaded by the caller); bucket b's first slot for this
// CTA is cursor[b * stride] (from the scan); every slot must lie in
// [0, bound).  The order of keys inside a bucket is not kept (the buckets
// are sorted afterwards).
template <class Tr>
__device__ __forceinline__ void scatter_range(const typename Tr::K *__restrict__ sk, const typename Tr::V *__restrict__ sv,
                                              typename Tr::K *__restrict__ dk, typename Tr::V *__restrict__ dv,
                                              int64_t lo, int64_t hi, ScatterSmem<Tr> &sm, int nsplit,
                                              const int64_t *cursor, int64_t stride, int64_t bound, LearnedState *st)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    using Ops = KeyOps<K>;
    constexpr int E = bucket_e<K>(), TILE = kThreads * E;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int bb = tid; bb < kBuckets; bb += kThreads) {
        sm.cursor[bb] = cursor[static_cast<int64_t>(bb) * stride];
        sm.tcnt[bb] = 0;
    }
    __syncthreads();
    for (int64_t base = lo; base < hi; base += TILE) {
        // Keep two tiles ahead in L2 (the first tile also covers itself).
        const int64_t pf = base == lo ? base : base + 2 * TILE;
        const int pn = base == lo ? 3 : 1;
        prefetch_tiles_l2(sk, pf, hi, TILE, pn);
        if constexpr (Tr::KV) prefetch_tiles_l2(sv, pf, hi, TILE, pn);
        const int cnt = static_cast<int>(hi - base < TILE ? hi - base : TILE);
        K key[E];
        V val[Tr::KV ? E : 1];
        int bk[E], rk[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int q = j * kThreads + tid;
            key[j] = q < cnt ? sk[base + q] : K(0);
            if constexpr (Tr::KV) val[j] = q < cnt ? sv[base + q] : 0;
        }
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int bb = bucket_of(sm.spl, Ops::to_s(key[j]));
            bk[j] = j * kThreads + tid < cnt ? (bb > nsplit ? nsplit : bb) : -1;
        }
#pragma unroll
        for (int j = 0; j < E; ++j) rk[j] = bk[j] >= 0 ? atomicAdd(&sm.tcnt[bk[j]], 1) : 0;
        __syncthreads();
        {  // exclusive scan of the tile's bucket counts (one thread per bucket)
            const int v = sm.tcnt[tid];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += x;
            }
            if (lane == 31) sm.wsum[warp] = incl;
            __syncthreads();
            int add = 0;
            for (int w = 0; w < warp; ++w) add += sm.wsum[w];
            sm.tstart[tid] = incl - v + add;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < E; ++j) {
            if (bk[j] < 0) continue;
            const int s = sm.tstart[bk[j]] + rk[j];
            sm.keys[s] = key[j];
            if constexpr (Tr::KV) sm.vals[s] = val[j];
            sm.bkt[s] = static_cast<unsigned char>(bk[j]);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int s = r * kThreads + tid;
            if (s >= cnt) continue;
            const int bb = sm.bkt[s];
            const long long d = sm.cursor[bb] + (s - sm.tstart[bb]);
            if (d < 0 || d >= bound) {
                st->status = -7;
                continue;
            }
            dk[d] = sm.keys[s];
            if constexpr (Tr::KV) dv[d] = sm.vals[s];
        }
        __syncthreads();
        sm.cursor[tid] += sm.tcnt[tid];
        sm.tcnt[tid] = 0;
        __syncthreads();
    }
}

// First level: CTA c of g scatters keys [c*n/g, (c+1)*n/g) from the caller's
// array into scratch.
template <class Tr>
__global__ void __launch_bounds__(kThreads) bucket_scatter_kernel(Args<typename Tr::K, typename Tr::V> a,
                                                                  LearnedBufs<typename Tr::K> lb, int nsplit)
{
    __shared__ ScatterSmem<Tr> sm;
    load_tree<typename Tr::K>(sm.spl, lb.splitters, nsplit);
    const int64_t c = blockIdx.x, g = gridDim.x, n = a.n;
    scatter_range<Tr>(a.keys[0], a.vals[0], a.keys[1], a.vals[1], c * n / g, (c + 1) * n / g, sm, nsplit, lb.cnt + c, g,
                      n, lb.st);
}

// ---------------------------------------------------------------------------
// Second bucket level (sample-sort style): each first-level bucket j, now in
// scratch at [bucket_off[j], bucket_off[j+1]), is split 256 ways again by its
// own splitters, from scratch back into the caller's array; the 65,536
// sub-buckets are then sorted by the plain method (most of them by the leaf
// kernel alone).  The passes give every CTA one chunk of kBucket2Chunk keys
// of one bucket, so large and small buckets get CTAs in proportion.
// ---------------------------------------------------------------------------

// Sub-splitters of bucket j (one CTA of 256 threads per bucket): 1024 keys
// sampled at jittered strides over the bucket, sorted with the Bitonic group
// network, every 4th kept -- the sampled form's rule, inside the bucket.
template <class K>
__global__ void __launch_bounds__(256) sub_splitter_kernel(const K *__restrict__ keys, LearnedBufs<K> lb)
{
    using Ops = KeyOps<K>;
    using S = typename Ops::S;
    constexpr int E = sizeof(S) == 8 ? 16 : 32, LE = sizeof(S) == 8 ? 4 : 5;
    constexpr int NG = kSketchN / E;  // threads of the sorting group
    __shared__ S sm[kSketchN + kSketchN / 16];
    const int t = threadIdx.x, j = blockIdx.x;
    const int64_t lo = lb.st->bucket_off[j], len = lb.st->bucket_off[j + 1] - lo;
    if (len <= 0) return;  // CTA-uniform: an empty bucket has no chunks either
    const int64_t stride = len / kSketchN;
    for (int i = t; i < kSketchN; i += 256) {
        const uint64_t h = mix64(static_cast<uint64_t>(lo) * 0x9E3779B97F4A7C15ull + i);
        const int64_t pos = (static_cast<int64_t>(i) * len) / kSketchN +
                            static_cast<int64_t>(h % static_cast<uint64_t>(stride > 0 ? stride : 1));
        sm[padk<S>(i)] = Ops::to_s(keys[lo + (pos < len ? pos : len - 1)]);
    }
    __syncthreads();
    if (t < NG) {
        S k[E];
        lay_load<E, LE, S>(k, sm, t, 0);
        group_bitonic_sort<E, LE, 10, S>(k, sm, t, 1, NG);
        group_sync(1, NG);
        lay_store<E, LE, S>(k, sm, t, 0);
    }
    __syncthreads();
    if (t < kBuckets - 1) lb.spl2[static_cast<int64_t>(j) * kBuckets + t] = sm[padk<S>(4 * (t + 1))];
}

// One CTA of kBuckets threads: chunks per bucket, their exclusive prefix
// (cbase[j] = the first chunk of bucket j, cbase[kBuckets] = all chunks).
template <class K>
__global__ void __launch_bounds__(kBuckets) chunk_plan_kernel(LearnedBufs<K> lb)
{
    __shared__ long long wsum[kBuckets / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t len = lb.st->bucket_off[t + 1] - lb.st->bucket_off[t];
    const long long v = len > 0 ? (len + kBucket2Chunk - 1) / kBucket2Chunk : 0;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    long long add = 0;
    for (int w = 0; w < warp; ++w) add += wsum[w];
    lb.cbase[t] = add + incl - v;
    if (t == kBuckets - 1) lb.cbase[kBuckets] = add + incl;
}

// The chunk of CTA b: bucket j (cbase[j] <= b < cbase[j+1]), its index c in
// the bucket, the bucket's chunk count, and the key range; false when b lies
// past the last chunk (the grid is an upper bound).
template <class K>
__device__ __forceinline__ bool chunk_of(const LearnedBufs<K> &lb, long long b, int &j, long long &c, long long &nch,
                                         int64_t &lo, int64_t &hi)
{
    if (b >= lb.cbase[kBuckets]) return false;
    int l = 0, r = kBuckets;  // largest j with cbase[j] <= b
    while (r - l > 1) {
        const int m = (l + r) >> 1;
        if (lb.cbase[m] <= b)
            l = m;
        else
            r = m;
    }
    j = l;
    c = b - lb.cbase[j];
    nch = lb.cbase[j + 1] - lb.cbase[j];
    const int64_t start = lb.st->bucket_off[j], end = lb.st->bucket_off[j + 1];
    lo = start + c * kBucket2Chunk;
    hi = lo + kBucket2Chunk < end ? lo + kBucket2Chunk : end;
    return true;
}

template <class Tr>
__global__ void __launch_bounds__(kThreads) bucket2_hist_kernel(const typename Tr::K *__restrict__ keys,
                                                                LearnedBufs<typename Tr::K> lb)
{
    __shared__ BucketSmem<Tr> sm;
    int j;
    long long c, nch;
    int64_t lo, hi;
    if (!chunk_of(lb, blockIdx.x, j, c, nch, lo, hi)) return;  // CTA-uniform
    load_tree<typename Tr::K>(sm.spl, lb.spl2 + static_cast<int64_t>(j) * kBuckets, kBuckets - 1);
    hist_range<Tr>(keys, lo, hi, sm, kBuckets - 1, lb.cnt2 + lb.cbase[j] * kBuckets + c, nch);
}

// One CTA of 1024 threads per bucket j: its (sub-bucket, chunk) counts become
// cursors, its sub-bucket starts go to off2[j*256 ...]; off2 ends with n.
template <class K>
__global__ void __launch_bounds__(1024) bucket2_scan_kernel(LearnedBufs<K> lb, int64_t n)
{
    const int j = blockIdx.x, t = threadIdx.x;
    const long long nch = lb.cbase[j + 1] - lb.cbase[j];
    const long long base = lb.st->bucket_off[j];
    int64_t *starts = lb.off2 + static_cast<int64_t>(j) * kBuckets;
    if (nch == 0) {  // CTA-uniform
        if (t < kBuckets) starts[t] = base;
    } else {
        scan_rows(lb.cnt2 + lb.cbase[j] * kBuckets, static_cast<int>(nch), base, starts);
    }
    if (j == 0 && t == 0) lb.off2[kLearnedBuckets2] = n;
}

template <class Tr>
__global__ void __launch_bounds__(kThreads) bucket2_scatter_kernel(Args<typename Tr::K, typename Tr::V> a,
                                                                   LearnedBufs<typename Tr::K> lb)
{
    __shared__ ScatterSmem<Tr> sm;
    int j;
    long long c, nch;
    int64_t lo, hi;
    if (!chunk_of(lb, blockIdx.x, j, c, nch, lo, hi)) return;  // CTA-uniform
    load_tree<typename Tr::K>(sm.spl, lb.spl2 + static_cast<int64_t>(j) * kBuckets, kBuckets - 1);
    scatter_range<Tr>(a.keys[1], a.vals[1], a.keys[0], a.vals[0], lo, hi, sm, kBuckets - 1,
                      lb.cnt2 + lb.cbase[j] * kBuckets + c, nch, a.n, lb.st);
}

}  // namespace qs
