// Kernel instantiation and launcher for the "f64" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
// Two partition tile variants (items per thread); the wide one is the default,
// the narrow one is chosen per call by QS_OPT_DRIVER_ITEMS (the autotuner).
using Tr = Traits<double, false, 8, 4096, 512>;
using TrN = Traits<double, false, 4, 4096, 512>;
// Minimum CTAs per SM: driver 3 (80 registers per thread), leaf 4 (64
// registers; the ALU-bound compare-exchange network hides its few spills --
// FP64 leaf kernel at 2^28: 9.07 ms at 2 CTAs, 8.36 at 3, 7.96 at 4; int32
// and key/value sorts equal at 3 and 4).
using L = Launcher<Tr, 3 * 256 / kDThreads, 4>;
using LN = Launcher<TrN, 3 * 256 / kDThreads, 4>;
}  // namespace

int launch_f64(const Args<Tr::K, Tr::V> &a, LaunchCfg &cfg)
{
    return cfg.items == TrN::E ? LN::launch(a, cfg) : L::launch(a, cfg);
}
KernelLimits limits_f64()
{
    KernelLimits l = L::limits();
    l.tile = TrN::T < Tr::T ? TrN::T : Tr::T;
    l.items_wide = Tr::E;
    l.items_narrow = TrN::E;
    l.items_default = Tr::E;
    return l;
}
int occupancy_f64(int which, int *bps) { return which == 2 ? LN::occ(0, bps) : L::occ(which, bps); }
int learned_f64(const Args<Tr::K, Tr::V> &a, const LearnedCall &lc, LaunchCfg &cfg) { return L::learned(a, lc, cfg); }

}  // namespace qs
