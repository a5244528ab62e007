// Kernel instantiation and launcher for the "f64" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
using Tr = Traits<double, false, 8, 4096, 512>;
using L = Launcher<Tr, 3 * 256 / kDThreads, 2>;  // driver CTAs per SM: register-bound at 80 per thread
}  // namespace

int launch_f64(const Args<Tr::K, Tr::V> &a, LaunchCfg &cfg) { return L::launch(a, cfg); }
KernelLimits limits_f64() { return L::limits(); }
int occupancy_f64(int which, int *bps) { return L::occ(which, bps); }
int learned_f64(const Args<Tr::K, Tr::V> &a, const LearnedCall &lc, LaunchCfg &cfg) { return L::learned(a, lc, cfg); }

}  // namespace qs
