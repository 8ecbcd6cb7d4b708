// Kernel instantiations for N = 2^LOGN, LOGN in { 7 8 9 10 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
#define KS_INST(N, R, C) \
  const LaunchTable &launch_table_##N##_##R##_##C() { return kern::Launch<N, R, C>::table(); }
KS_INST(7, 3, 0)
KS_INST(7, 2, 0)
KS_INST(7, 4, 0)
KS_INST(8, 3, 0)
KS_INST(8, 2, 0)
KS_INST(8, 4, 0)
KS_INST(9, 3, 0)
KS_INST(9, 2, 0)
KS_INST(9, 4, 0)
KS_INST(10, 3, 0)
KS_INST(10, 2, 0)
KS_INST(10, 4, 0)
#undef KS_INST
}  // namespace ks
