// Kernel instantiations for N = 2^LOGN, LOGN in { 7 8 9 10 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_7() { return kern::Launch<7>::table(); }
const LaunchTable &launch_table_8() { return kern::Launch<8>::table(); }
const LaunchTable &launch_table_9() { return kern::Launch<9>::table(); }
const LaunchTable &launch_table_10() { return kern::Launch<10>::table(); }
}  // namespace ks
