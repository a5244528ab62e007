// Kernel instantiation and launcher for the "kv" element kind.
#include "qs_launch.cuh"

namespace qs {

namespace {
using Tr = Traits<int32_t, true, 4, 4096, 512>;
using L = Launcher<Tr, 3 * 256 / kDThreads, 2>;  // driver CTAs per SM: register-bound at 80 per thread
}  // namespace

int launch_kv(const Args<Tr::K, Tr::V> &a, LaunchCfg &cfg) { return L::launch(a, cfg); }
KernelLimits limits_kv() { return L::limits(); }
int occupancy_kv(int which, int *bps) { return L::occ(which, bps); }

}  // namespace qs
