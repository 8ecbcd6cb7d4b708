// Kernel instantiations for N = 2^LOGN, LOGN in { 13 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_13_3() { return kern::Launch<13, 3>::table(); }
const LaunchTable &launch_table_13_2() { return kern::Launch<13, 2>::table(); }
const LaunchTable &launch_table_13_4() { return kern::Launch<13, 4>::table(); }
}  // namespace ks
