// Kernel instantiations for N = 2^LOGN, LOGN in { 11 12 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_11_3() { return kern::Launch<11, 3>::table(); }
const LaunchTable &launch_table_11_2() { return kern::Launch<11, 2>::table(); }
const LaunchTable &launch_table_11_4() { return kern::Launch<11, 4>::table(); }
const LaunchTable &launch_table_12_3() { return kern::Launch<12, 3>::table(); }
const LaunchTable &launch_table_12_2() { return kern::Launch<12, 2>::table(); }
const LaunchTable &launch_table_12_4() { return kern::Launch<12, 4>::table(); }
}  // namespace ks
