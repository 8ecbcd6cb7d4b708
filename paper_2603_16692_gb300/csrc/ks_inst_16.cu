// Kernel instantiations for N = 2^LOGN, LOGN in { 16 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_16_3() { return kern::Launch<16, 3>::table(); }
const LaunchTable &launch_table_16_2() { return kern::Launch<16, 2>::table(); }
const LaunchTable &launch_table_16_4() { return kern::Launch<16, 4>::table(); }
}  // namespace ks
