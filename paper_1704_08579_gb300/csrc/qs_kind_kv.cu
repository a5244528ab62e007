// Kernel instantiation and launcher for the "kv" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
// Three partition tile variants (items per thread), chosen per call by
// QS_OPT_DRIVER_ITEMS (the autotuner): wide and narrow prefetched tiles, and
// the register tile.  Sorts default to the register tile (2^28: 12.11 against 13.66 ms of partition passes),
// partitions to the wide tile (the register tile's partition lacks the
// early published aggregates of prefetched tiles: 1.72 against 1.01 ms).
using Tr = Traits<int32_t, true, 4, 16384, 512>;
using TrN = Traits<int32_t, true, 2, 16384, 512>;
// Register tile: 20 keys and values per thread on 128-thread CTAs (2560 pairs, 20 KB), loaded straight
// into registers, 6 CTAs per SM (80 registers); 32 pairs on 256 threads at 2 CTAs per SM: 12.83 ms, 16
// pairs on 128 threads at 8 per SM: 11.91 ms (but 16 is the wide tile's selector value).
using TrX = Traits<int32_t, true, 5, 16384, 512, false, 128>;
// Minimum CTAs per SM of the persistent partition kernel: 3 (80 registers
// per thread).  The leaf kernel runs one 1024-thread CTA per SM.
using L = Launcher<Tr, 3 * 256 / kDThreads>;
using LN = Launcher<TrN, 3 * 256 / kDThreads>;
using LX = Launcher<TrX, 6>;
}  // namespace

int launch_kv(const Args<Tr::K, Tr::V> &a, LaunchCfg &cfg)
{
    if (cfg.items == TrX::E) return LX::launch(a, cfg);
    return cfg.items == TrN::E ? LN::launch(a, cfg) : L::launch(a, cfg);
}
KernelLimits limits_kv()
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
int occupancy_kv(int which, int *bps)
{
    return which == 3 ? LX::occ(0, bps) : which == 2 ? LN::occ(0, bps) : L::occ(which, bps);
}

}  // namespace qs
