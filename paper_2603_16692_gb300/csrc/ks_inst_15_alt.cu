// Kernel instantiations for N = 2^LOGN, LOGN in { 15 }, radix 8, 4 and 16, alternative column tile.
#include "ks_kern.cuh"

namespace ks {
#define KS_INST(N, R, C) \
  const LaunchTable &launch_table_##N##_##R##_##C() { return kern::Launch<N, R, C>::table(); }
KS_INST(15, 3, 1)
KS_INST(15, 2, 1)
KS_INST(15, 4, 1)
#undef KS_INST
}  // namespace ks
