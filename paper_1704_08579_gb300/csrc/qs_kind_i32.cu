// Kernel instantiation and launcher for the "i32" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
using Tr = Traits<int32_t, false, 8, 8192, 512>;
using L = Launcher<Tr, 3 * 256 / kDThreads, 2>;  // driver CTAs per SM: register-bound at 80 per thread
}  // namespace

int launch_i32(const Args<Tr::K, Tr::V> &a, LaunchCfg &cfg) { return L::launch(a, cfg); }
KernelLimits limits_i32() { return L::limits(); }
int occupancy_i32(int which, int *bps) { return L::occ(which, bps); }
int learned_i32(const Args<Tr::K, Tr::V> &a, const LearnedCall &lc, LaunchCfg &cfg) { return L::learned(a, lc, cfg); }

}  // namespace qs
