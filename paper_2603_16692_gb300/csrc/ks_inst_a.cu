// Kernel instantiations for N = 2^LOGN, LOGN in { 1 2 3 4 5 6 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_1() { return kern::Launch<1>::table(); }
const LaunchTable &launch_table_2() { return kern::Launch<2>::table(); }
const LaunchTable &launch_table_3() { return kern::Launch<3>::table(); }
const LaunchTable &launch_table_4() { return kern::Launch<4>::table(); }
const LaunchTable &launch_table_5() { return kern::Launch<5>::table(); }
const LaunchTable &launch_table_6() { return kern::Launch<6>::table(); }
}  // namespace ks
