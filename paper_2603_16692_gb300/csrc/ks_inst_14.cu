// Kernel instantiations for N = 2^LOGN, LOGN in { 14 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_14() { return kern::Launch<14>::table(); }
}  // namespace ks
