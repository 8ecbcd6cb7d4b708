// Kernel instantiations for N = 2^LOGN, LOGN in { 15 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_15() { return kern::Launch<15>::table(); }
}  // namespace ks
