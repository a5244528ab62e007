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

// Bucket of sort-space key s among nsplit (<= 255) sorted splitters held in
// shared memory, padded to 255 with the largest key: number of splitters <= s.
template <class S>
__device__ __forceinline__ int bucket_of(const S *spl, S s)
{
    int pos = 0;
#pragma unroll
    for (int step = 128; step >= 1; step >>= 1)
        if (!(s < spl[pos + step - 1])) pos += step;
    return pos;
}

template <class Tr>
struct BucketSmem {
    typename KeyOps<typename Tr::K>::S spl[255];
    int hist[kWarps][kBuckets];
};

// Loads the splitters into shared memory, padding the unused slots with the
// largest key.  Only a key equal to the largest key can count a pad; such a
// key belongs to the last bucket anyway, so callers clamp the bucket to nsplit.
template <class Tr>
__device__ __forceinline__ void load_splitters(typename KeyOps<typename Tr::K>::S *spl, const LearnedBufs<typename Tr::K> &lb,
                                               int nsplit)
{
    using Ops = KeyOps<typename Tr::K>;
    for (int i = threadIdx.x; i < 255; i += kThreads) spl[i] = i < nsplit ? lb.splitters[i] : Ops::s_largest();
}

template <class Tr>
__global__ void __launch_bounds__(kThreads) bucket_hist_kernel(const typename Tr::K *__restrict__ keys, int64_t n,
                                                               LearnedBufs<typename Tr::K> lb, int nsplit)
{
    using Ops = KeyOps<typename Tr::K>;
    __shared__ BucketSmem<Tr> sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    load_splitters<Tr>(sm.spl, lb, nsplit);
    for (int i = tid; i < kWarps * kBuckets; i += kThreads) (&sm.hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t c = blockIdx.x, g = gridDim.x;
    const int64_t lo = c * n / g, hi = (c + 1) * n / g;
    for (int64_t base = lo; base < hi; base += kThreads) {
        const int64_t i = base + tid;
        const bool ok = i < hi;
        int b = ok ? bucket_of(sm.spl, Ops::to_s(keys[i])) : -1;
        if (b > nsplit) b = nsplit;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        if (ok && lane == leader) sm.hist[warp][b] += __popc(peers);
    }
    __syncthreads();
    for (int b = tid; b < kBuckets; b += kThreads) {
        int s = 0;
        for (int w = 0; w < kWarps; ++w) s += sm.hist[w][b];
        lb.cnt[static_cast<int64_t>(b) * g + c] = s;
    }
}

// One CTA: exclusive scan over (bucket, cta) counts in bucket-major order.
static __global__ void __launch_bounds__(1024) bucket_scan_kernel(int64_t *__restrict__ cnt, int ctas, LearnedState *st,
                                                           int nsplit, int64_t n, int64_t bound)
{
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const int64_t total = static_cast<int64_t>(kBuckets) * ctas;
    const int64_t per = (total + 1023) / 1024;
    const int64_t a = t * per, e = a + per < total ? a + per : total;
    long long s = 0;
    for (int64_t i = a; i < e; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the 1024 partial sums
        const long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = t > 0 ? part[t - 1] : 0;
    for (int64_t i = a; i < e; ++i) {
        const long long v = cnt[i];
        cnt[i] = run;
        if (i % ctas == 0) st->bucket_off[i / ctas] = run;
        run += v;
    }
    __syncthreads();
    if (t == 0) {
        st->bucket_off[nsplit + 1] = n;
        unsigned long long mx = 0, over = 0, dev = 0;
        for (int b = 0; b <= nsplit; ++b) {
            const unsigned long long sz = static_cast<unsigned long long>(st->bucket_off[b + 1] - st->bucket_off[b]);
            mx = sz > mx ? sz : mx;
            over += sz > static_cast<unsigned long long>(bound) ? 1 : 0;
            const long long d = static_cast<long long>(sz) * (nsplit + 1) - n;  // vs the even share n/(nsplit+1)
            dev += static_cast<unsigned long long>(d < 0 ? -d : d);
        }
        st->bucket_max = mx;
        st->bucket_over = over;
        st->bucket_dev = dev;
    }
}

static_assert(kThreads == kBuckets, "one thread per bucket in the scatter's per-tile bookkeeping");

template <class Tr>
struct ScatterSmem {
    typename KeyOps<typename Tr::K>::S spl[255];
    typename Tr::K keys[kThreads * 8];
    typename Tr::V vals[Tr::KV ? kThreads * 8 : 1];
    unsigned char bkt[kThreads * 8];
    int tcnt[kBuckets];
    int tstart[kBuckets];
    long long cursor[kBuckets];
    int wsum[kWarps];
};

template <class Tr>
__global__ void __launch_bounds__(kThreads) bucket_scatter_kernel(Args<typename Tr::K, typename Tr::V> a,
                                                                  LearnedBufs<typename Tr::K> lb, int nsplit)
{
    using K = typename Tr::K;
    using V = typename Tr::V;
    using Ops = KeyOps<K>;
    constexpr int E = 8, TILE = kThreads * E;
    __shared__ ScatterSmem<Tr> sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = blockIdx.x, g = gridDim.x, n = a.n;
    const int64_t lo = c * n / g, hi = (c + 1) * n / g;
    load_splitters<Tr>(sm.spl, lb, nsplit);
    for (int b = tid; b < kBuckets; b += kThreads) {
        sm.cursor[b] = lb.cnt[static_cast<int64_t>(b) * g + c];
        sm.tcnt[b] = 0;
    }
    __syncthreads();
    const K *__restrict__ sk = a.keys[0];
    const V *__restrict__ sv = a.vals[0];
    K *__restrict__ dk = a.keys[1];
    V *__restrict__ dv = a.vals[1];
    for (int64_t base = lo; base < hi; base += TILE) {
        const int cnt = static_cast<int>(hi - base < TILE ? hi - base : TILE);
        K key[E];
        V val[E];
        int bk[E], rk[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int q = j * kThreads + tid;
            const bool ok = q < cnt;
            key[j] = ok ? sk[base + q] : K(0);
            if constexpr (Tr::KV) val[j] = ok ? sv[base + q] : 0;
            int b = ok ? bucket_of(sm.spl, Ops::to_s(key[j])) : -1;
            if (b > nsplit) b = nsplit;
            bk[j] = b;
            const unsigned peers = __match_any_sync(0xffffffffu, b);
            const int leader = __ffs(peers) - 1;
            int r0 = 0;
            if (ok && lane == leader) r0 = atomicAdd(&sm.tcnt[b], __popc(peers));
            r0 = __shfl_sync(0xffffffffu, r0, leader);
            rk[j] = r0 + __popc(peers & ((1u << lane) - 1u));
        }
        __syncthreads();
        // exclusive scan of the tile's bucket counts
        {
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
        for (int s = tid; s < cnt; s += kThreads) {
            const int b = sm.bkt[s];
            const long long d = sm.cursor[b] + (s - sm.tstart[b]);
            if (d < 0 || d >= n) {
                lb.st->status = -7;
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

}  // namespace qs
