// Kernel instantiations for N = 2^LOGN, LOGN in { 15 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_15_3() { return kern::Launch<15, 3>::table(); }
const LaunchTable &launch_table_15_2() { return kern::Launch<15, 2>::table(); }
const LaunchTable &launch_table_15_4() { return kern::Launch<15, 4>::table(); }
}  // namespace ks
