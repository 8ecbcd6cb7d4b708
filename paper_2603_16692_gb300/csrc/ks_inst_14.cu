// Kernel instantiations for N = 2^LOGN, LOGN in { 14 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_14_3() { return kern::Launch<14, 3>::table(); }
const LaunchTable &launch_table_14_2() { return kern::Launch<14, 2>::table(); }
const LaunchTable &launch_table_14_4() { return kern::Launch<14, 4>::table(); }
}  // namespace ks
