// Kernel instantiations for N = 2^LOGN, LOGN in { 1 2 3 4 5 6 }, radix 8, 4 and 16.
#include "ks_kern.cuh"

namespace ks {
#define KS_INST(N, R, C) \
  const LaunchTable &launch_table_##N##_##R##_##C() { return kern::Launch<N, R, C>::table(); }
KS_INST(1, 3, 0)
KS_INST(1, 2, 0)
KS_INST(1, 4, 0)
KS_INST(2, 3, 0)
KS_INST(2, 2, 0)
KS_INST(2, 4, 0)
KS_INST(3, 3, 0)
KS_INST(3, 2, 0)
KS_INST(3, 4, 0)
KS_INST(4, 3, 0)
KS_INST(4, 2, 0)
KS_INST(4, 4, 0)
KS_INST(5, 3, 0)
KS_INST(5, 2, 0)
KS_INST(5, 4, 0)
KS_INST(6, 3, 0)
KS_INST(6, 2, 0)
KS_INST(6, 4, 0)
#undef KS_INST
}  // namespace ks
