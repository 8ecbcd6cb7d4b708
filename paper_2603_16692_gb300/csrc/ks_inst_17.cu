// Kernel instantiations for N = 2^LOGN, LOGN in { 17 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
#define KS_INST(N, R, C) \
  const LaunchTable &launch_table_##N##_##R##_##C() { return kern::Launch<N, R, C>::table(); }
KS_INST(17, 3, 0)
KS_INST(17, 2, 0)
KS_INST(17, 4, 0)
#undef KS_INST
}  // namespace ks
