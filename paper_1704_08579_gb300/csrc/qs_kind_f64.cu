// Kernel instantiation and launcher for the "f64" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
// Three partition tile variants (items per thread), chosen per call by
// QS_OPT_DRIVER_ITEMS (the autotuner): wide and narrow prefetched tiles, and
// the register tile.  Sorts default to the register tile (2^28: 11.18 against 12.97 ms of partition passes),
// partitions to the wide tile (the register tile's partition lacks the
// early published aggregates of prefetched tiles: 1.72 against 1.01 ms).
using Tr = Traits<double, false, 8, 16384, 512>;
using TrN = Traits<double, false, 4, 16384, 512>;
// Register tile: 20 keys per thread on 128-thread CTAs (2560 keys, 20 KB), loaded straight into
// registers, 6 CTAs per SM (80 registers).  At 2^28 keys, the partition passes of other shapes: 32 keys
// on 256 threads at 2 CTAs per SM 12.00 ms; on 128 threads, 32 keys at 4 per SM 11.70, 24 at 5 11.32,
// 16 at 8 11.47, 20 at 6 11.18 (this one): smaller tiles on more CTAs overlap more of each tile's
// fixed chain of claims, barriers and release, until the chains per key outgrow the overlap.
using TrX = Traits<double, false, 10, 16384, 512, false, 128>;
// Minimum CTAs per SM of the persistent partition kernel: 3 (80 registers
// per thread).  The leaf kernel runs one 1024-thread CTA per SM.
using L = Launcher<Tr, 3 * 256 / kDThreads>;
using LN = Launcher<TrN, 3 * 256 / kDThreads>;
using LX = Launcher<TrX, 6>;
}  // namespace

int launch_f64(const Args<Tr::K, Tr::V> &a, LaunchCfg &cfg)
{
    if (cfg.items == TrX::E) return LX::launch(a, cfg);
    return cfg.items == TrN::E ? LN::launch(a, cfg) : L::launch(a, cfg);
}
KernelLimits limits_f64()
{
    KernelLimits l = L::limits();
    l.tile = TrN::T < Tr::T ? TrN::T : Tr::T;
    l.items_wide = Tr::E;
    l.items_narrow = TrN::E;
    l.items_xwide = TrX::E;
    l.items_default = TrX::E;
    l.items_default_part = Tr::E;
    return l;
}
int occupancy_f64(int which, int *bps)
{
    return which == 3 ? LX::occ(0, bps) : which == 2 ? LN::occ(0, bps) : L::occ(which, bps);
}
int learned_f64(const Args<Tr::K, Tr::V> &a, const LearnedCall &lc, LaunchCfg &cfg) { return L::learned(a, lc, cfg); }

}  // namespace qs
