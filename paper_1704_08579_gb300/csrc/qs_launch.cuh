// Host-side launcher of one element kind: setup kernel, persistent partition
// kernel, leaf kernel, all on the caller's stream.
#pragma once

#include <cuda_runtime.h>

#include "qs_driver.cuh"
#include "qs_leaf.cuh"
#include "qs_learned.cuh"

namespace qs {

template <class Tr, int DriverMin>
struct Launcher {
    using K = typename Tr::K;
    using V = typename Tr::V;
    // The leaf kernel depends only on the key kind and the leaf sizes: the
    // partition tile variants of a kind share one instantiation.
    using LTr = Traits<K, Tr::KV, 1, Tr::LEAF, Tr::SMALL>;
    static constexpr size_t kDriverSmem = sizeof(DriverSmem<Tr>);

    static KernelLimits limits()
    {
        KernelLimits l;
        l.leaf_max = Tr::MID;
        l.leaf_default = Tr::LEAF;
        l.small_max = Tr::SMALL;
        l.tile = Tr::T;
        l.driver_smem = kDriverSmem;
        l.leaf_smem = sizeof(LeafSmem<LTr>) + LeafCfg<LTr>::kDynSmem;
        return l;
    }
    static int prepare()
    {
        static int done = 0;
        static int rc = 0;
        if (!done) {
            rc = cudaFuncSetAttribute(driver_kernel<Tr, DriverMin>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(kDriverSmem));
            if (rc == 0)
                rc = cudaFuncSetAttribute(leaf_kernel<LTr, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(LeafCfg<LTr>::kDynSmem));
            if (rc == 0)
                rc = cudaFuncSetAttribute(leaf_kernel<LTr, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(LeafCfg<LTr>::kDynSmem));
            done = 1;
        }
        return rc;
    }
    static int occ(int which, int *bps)
    {
        int rc = prepare();
        if (rc) return rc;
        if (which == 0)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, driver_kernel<Tr, DriverMin>, Tr::DT,
                                                                 kDriverSmem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, leaf_kernel<LTr, false>, kLThreads,
                                                             LeafCfg<LTr>::kDynSmem);
    }
    static int launch(const Args<K, V> &a, LaunchCfg &cfg)
    {
        int rc = prepare();
        if (rc) return rc;
        cudaStream_t s = static_cast<cudaStream_t>(cfg.stream);
        cudaEvent_t *ev = reinterpret_cast<cudaEvent_t *>(cfg.ev);
        if (cfg.profile) cudaEventRecord(ev[0], s);
        setup_kernel<Tr><<<1, kThreads, 0, s>>>(a);
        if (a.seg_off) {
            const long long blocks = (a.nseg + kWarps - 1) / kWarps;
            setup_segments_kernel<Tr><<<static_cast<int>(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), kThreads, 0, s>>>(a);
        }
        if (cfg.profile) cudaEventRecord(ev[1], s);
        if (a.partition_only || a.seg_off || a.n > a.leaf_max)
            driver_kernel<Tr, DriverMin><<<cfg.grid_driver, Tr::DT, kDriverSmem, s>>>(a);
        if (cfg.profile) cudaEventRecord(ev[2], s);
        if (!a.partition_only) {
            // Parts above LEAF are listed only when the threshold allows them.
            if (a.leaf_max > LTr::LEAF)
                leaf_kernel<LTr, true><<<cfg.grid_leaf, kLThreads, LeafCfg<LTr>::kDynSmem, s>>>(a);
            else
                leaf_kernel<LTr, false><<<cfg.grid_leaf, kLThreads, LeafCfg<LTr>::kDynSmem, s>>>(a);
        }
        if (cfg.profile) cudaEventRecord(ev[3], s);
        return static_cast<int>(cudaGetLastError());
    }
    // Sketch / bucket pass / learned sort (keys only).
    static int learned(const Args<K, V> &a, const LearnedCall &lc, LaunchCfg &cfg)
    {
        int rc = prepare();
        if (rc) return rc;
        cudaStream_t s = static_cast<cudaStream_t>(cfg.stream);
        const LearnedBufs<K> lb = bufs_of<K>(lc.p);
        sketch_kernel<K><<<1, 256, 0, s>>>(a.keys[0], a.n, lb, lc.sketch_out, lc.minmax_out, static_cast<K *>(lc.sample_out));
        if (lc.op == kOpSketch) return static_cast<int>(cudaGetLastError());
        int nsplit = 255;
        if (lc.op == kOpBucket) {
            nsplit = lc.nsplit;
            splitters_from_keys_kernel<K><<<1, 256, 0, s>>>(static_cast<const K *>(lc.user_spl), nsplit, lb);
        } else {
            splitter_kernel<K><<<1, 256, 0, s>>>(lc.params, lb);
        }
        bucket_hist_kernel<Tr><<<lc.ctas, kThreads, 0, s>>>(a.keys[0], a.n, lb, nsplit);
        bucket_scan_kernel<<<1, 1024, 0, s>>>(lb.cnt, lc.ctas, lb.st, nsplit, a.n, lc.bound);
        bucket_scatter_kernel<Tr><<<lc.ctas, kThreads, 0, s>>>(a, lb, nsplit);
        if (lc.op == kOpBucket) return static_cast<int>(cudaGetLastError());
        Args<K, V> a2 = a;
        if (lc.levels == 2) {
            // Second level: every bucket split 256 ways by its own sampled
            // splitters, from scratch back into the caller's array; then the
            // 65,536 sub-buckets are sorted by the plain method.
            sub_splitter_kernel<K><<<kBuckets, 256, 0, s>>>(a.keys[1], lb);
            chunk_plan_kernel<K><<<1, kBuckets, 0, s>>>(lb);
            bucket2_hist_kernel<Tr><<<lc.ctas2, kThreads, 0, s>>>(a.keys[1], lb);
            bucket2_scan_kernel<K><<<kBuckets, 1024, 0, s>>>(lb, a.n);
            bucket2_scatter_kernel<Tr><<<lc.ctas2, kThreads, 0, s>>>(a, lb);
            a2.seg_off = lb.off2;
            a2.nseg = kLearnedBuckets2;
            a2.seg_src = 0;
        } else {
            // Every bucket is sorted by the plain method, straight from scratch.
            a2.seg_off = lb.st->bucket_off;
            a2.nseg = kBuckets;
            a2.seg_src = 1;
        }
        return launch(a2, cfg);
    }
};

}  // namespace qs
