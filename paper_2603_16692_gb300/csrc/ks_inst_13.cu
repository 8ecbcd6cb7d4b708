// Kernel instantiations for N = 2^LOGN, LOGN in { 13 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_13() { return kern::Launch<13>::table(); }
}  // namespace ks
