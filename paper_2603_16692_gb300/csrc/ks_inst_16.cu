// Kernel instantiations for N = 2^LOGN, LOGN in { 16 }.
#include "ks_kern.cuh"

namespace ks {
const LaunchTable &launch_table_16() { return kern::Launch<16>::table(); }
}  // namespace ks
