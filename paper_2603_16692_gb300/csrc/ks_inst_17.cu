// Kernel instantiations for N = 2^LOGN, LOGN in { 17 }, radix 8 and 4.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_17_3() { return kern::Launch<17, 3>::table(); }
const LaunchTable &launch_table_17_2() { return kern::Launch<17, 2>::table(); }
}  // namespace ks
