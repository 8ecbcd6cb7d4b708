// Kernel instantiations for N = 2^LOGN, LOGN in { 1 2 3 4 5 6 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_1_3() { return kern::Launch<1, 3>::table(); }
const LaunchTable &launch_table_1_2() { return kern::Launch<1, 2>::table(); }
const LaunchTable &launch_table_1_4() { return kern::Launch<1, 4>::table(); }
const LaunchTable &launch_table_2_3() { return kern::Launch<2, 3>::table(); }
const LaunchTable &launch_table_2_2() { return kern::Launch<2, 2>::table(); }
const LaunchTable &launch_table_2_4() { return kern::Launch<2, 4>::table(); }
const LaunchTable &launch_table_3_3() { return kern::Launch<3, 3>::table(); }
const LaunchTable &launch_table_3_2() { return kern::Launch<3, 2>::table(); }
const LaunchTable &launch_table_3_4() { return kern::Launch<3, 4>::table(); }
const LaunchTable &launch_table_4_3() { return kern::Launch<4, 3>::table(); }
const LaunchTable &launch_table_4_2() { return kern::Launch<4, 2>::table(); }
const LaunchTable &launch_table_4_4() { return kern::Launch<4, 4>::table(); }
const LaunchTable &launch_table_5_3() { return kern::Launch<5, 3>::table(); }
const LaunchTable &launch_table_5_2() { return kern::Launch<5, 2>::table(); }
const LaunchTable &launch_table_5_4() { return kern::Launch<5, 4>::table(); }
const LaunchTable &launch_table_6_3() { return kern::Launch<6, 3>::table(); }
const LaunchTable &launch_table_6_2() { return kern::Launch<6, 2>::table(); }
const LaunchTable &launch_table_6_4() { return kern::Launch<6, 4>::table(); }
}  // namespace ks
