// Kernel instantiations for N = 2^LOGN, LOGN in { 17 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_17() { return kern::Launch<17>::table(); }
}  // namespace ks
