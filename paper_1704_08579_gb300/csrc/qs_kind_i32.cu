// Kernel instantiation and launcher for the "i32" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
// Two partition tile variants (items per thread), chosen per call by
// QS_OPT_DRIVER_ITEMS (the autotuner): the register tile -- 32 keys per
// thread, 32 KB loaded straight into registers with 16-byte loads, the next
// tile prefetched into L2, 4 CTAs per SM (64 registers) -- the sorts'
// default (2^28 keys: 7.05 ms of partition passes against 8.30 for the
// prefetched 32-key tile it replaced; the same tile on 512-thread CTAs, 64
// KB at 2 CTAs per SM: 7.69 ms), and the narrow prefetched tile (16
// keys, TMA double buffer, 4 CTAs per SM), the partitions' default.  The
// leaf kernel runs one 1024-thread CTA per SM.
using Tr = Traits<int32_t, false, 8, 32768, 512, false>;
using TrN = Traits<int32_t, false, 4, 32768, 512>;
using L = Launcher<Tr, 4>;
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
    l.items_xwide = 0;  // the 32-key variant is itself a register tile
    l.items_default = Tr::E;
    l.items_default_part = TrN::E;
    return l;
}
int occupancy_i32(int which, int *bps) { return which == 2 ? LN::occ(0, bps) : L::occ(which == 3 ? 0 : which, bps); }
int learned_i32(const Args<Tr::K, Tr::V> &a, const LearnedCall &lc, LaunchCfg &cfg) { return L::learned(a, lc, cfg); }

}  // namespace qs
