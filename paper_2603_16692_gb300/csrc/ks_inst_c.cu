// Kernel instantiations for N = 2^LOGN, LOGN in { 11 12 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_11() { return kern::Launch<11>::table(); }
const LaunchTable &launch_table_12() { return kern::Launch<12>::table(); }
}  // namespace ks
