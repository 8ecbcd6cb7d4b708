// Kernel instantiations for N = 2^LOGN, LOGN in { 7 8 9 10 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_7_3() { return kern::Launch<7, 3>::table(); }
const LaunchTable &launch_table_7_2() { return kern::Launch<7, 2>::table(); }
const LaunchTable &launch_table_7_4() { return kern::Launch<7, 4>::table(); }
const LaunchTable &launch_table_8_3() { return kern::Launch<8, 3>::table(); }
const LaunchTable &launch_table_8_2() { return kern::Launch<8, 2>::table(); }
const LaunchTable &launch_table_8_4() { return kern::Launch<8, 4>::table(); }
const LaunchTable &launch_table_9_3() { return kern::Launch<9, 3>::table(); }
const LaunchTable &launch_table_9_2() { return kern::Launch<9, 2>::table(); }
const LaunchTable &launch_table_9_4() { return kern::Launch<9, 4>::table(); }
const LaunchTable &launch_table_10_3() { return kern::Launch<10, 3>::table(); }
const LaunchTable &launch_table_10_2() { return kern::Launch<10, 2>::table(); }
const LaunchTable &launch_table_10_4() { return kern::Launch<10, 4>::table(); }
}  // namespace ks
