// Kernel instantiations for N = 2^LOGN, LOGN in { 17 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_17_3() { return kern::Launch<17, 3>::table(); }
const LaunchTable &launch_table_17_2() { return kern::Launch<17, 2>::table(); }
const LaunchTable &launch_table_17_4() { return kern::Launch<17, 4>::table(); }
}  // namespace ks
