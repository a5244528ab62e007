// Kernel instantiation and launcher for the "i32" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
// Two partition tile variants (items per thread), chosen per call by
// QS_OPT_DRIVER_ITEMS (the autotuner).  Sorts default to the wide one (2^28
// keys: 8.08 ms of partition passes against 8.39 for the narrow one at 4 CTAs
// per SM); partitions keep the narrow one.
using Tr = Traits<int32_t, false, 8, 32768, 512>;
using TrN = Traits<int32_t, false, 4, 32768, 512>;
// Minimum CTAs per SM of the persistent partition kernel: 3 (80 registers
// per thread); the narrow int32 tile 4 (64 registers).  The leaf kernel
// runs one 1024-thread CTA per SM.
using L = Launcher<Tr, 3 * 256 / kDThreads>;
using LN = Launcher<TrN, 4>;
}  // namespace

int launch_i32(const Args<Tr::K, Tr::V> &a, LaunchCfg &cfg)
{
    return cfg.items == TrN::E ? LN::launch(a, cfg) : L::launch(a, cfg);
}
KernelLimits limits_i32()
{
    KernelLimits l = L::limits();
    l.tile = TrN::T < Tr::T ? TrN::T : Tr::T;
    l.items_wide = Tr::E;
    l.items_narrow = TrN::E;
    l.items_xwide = 0;  // a register tile would need 64 keys per thread
    l.items_default = Tr::E;
    l.items_default_part = TrN::E;
    return l;
}
int occupancy_i32(int which, int *bps) { return which == 2 ? LN::occ(0, bps) : L::occ(which == 3 ? 0 : which, bps); }
int learned_i32(const Args<Tr::K, Tr::V> &a, const LearnedCall &lc, LaunchCfg &cfg) { return L::learned(a, lc, cfg); }

}  // namespace qs
