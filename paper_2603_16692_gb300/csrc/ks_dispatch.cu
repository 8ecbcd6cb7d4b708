// Run-time selection of the per-N kernel launchers.
#include <mutex>
#include <unordered_map>

#include "ks_internal.h"

namespace ks {
const LaunchTable &launch_table_1_3_0();
const LaunchTable &launch_table_1_2_0();
const LaunchTable &launch_table_1_4_0();
const LaunchTable &launch_table_2_3_0();
const LaunchTable &launch_table_2_2_0();
const LaunchTable &launch_table_2_4_0();
const LaunchTable &launch_table_3_3_0();
const LaunchTable &launch_table_3_2_0();
const LaunchTable &launch_table_3_4_0();
const LaunchTable &launch_table_4_3_0();
const LaunchTable &launch_table_4_2_0();
const LaunchTable &launch_table_4_4_0();
const LaunchTable &launch_table_5_3_0();
const LaunchTable &launch_table_5_2_0();
const LaunchTable &launch_table_5_4_0();
const LaunchTable &launch_table_6_3_0();
const LaunchTable &launch_table_6_2_0();
const LaunchTable &launch_table_6_4_0();
const LaunchTable &launch_table_7_3_0();
const LaunchTable &launch_table_7_2_0();
const LaunchTable &launch_table_7_4_0();
const LaunchTable &launch_table_8_3_0();
const LaunchTable &launch_table_8_2_0();
const LaunchTable &launch_table_8_4_0();
const LaunchTable &launch_table_9_3_0();
const LaunchTable &launch_table_9_2_0();
const LaunchTable &launch_table_9_4_0();
const LaunchTable &launch_table_10_3_0();
const LaunchTable &launch_table_10_2_0();
const LaunchTable &launch_table_10_4_0();
const LaunchTable &launch_table_11_3_0();
const LaunchTable &launch_table_11_2_0();
const LaunchTable &launch_table_11_4_0();
const LaunchTable &launch_table_12_3_0();
const LaunchTable &launch_table_12_2_0();
const LaunchTable &launch_table_12_4_0();
const LaunchTable &launch_table_13_3_0();
const LaunchTable &launch_table_13_3_1();
const LaunchTable &launch_table_13_2_0();
const LaunchTable &launch_table_13_2_1();
const LaunchTable &launch_table_13_4_0();
const LaunchTable &launch_table_13_4_1();
const LaunchTable &launch_table_14_3_0();
const LaunchTable &launch_table_14_3_1();
const LaunchTable &launch_table_14_2_0();
const LaunchTable &launch_table_14_2_1();
const LaunchTable &launch_table_14_4_0();
const LaunchTable &launch_table_14_4_1();
const LaunchTable &launch_table_15_3_0();
const LaunchTable &launch_table_15_3_1();
const LaunchTable &launch_table_15_2_0();
const LaunchTable &launch_table_15_2_1();
const LaunchTable &launch_table_15_4_0();
const LaunchTable &launch_table_15_4_1();
const LaunchTable &launch_table_16_3_0();
const LaunchTable &launch_table_16_3_1();
const LaunchTable &launch_table_16_2_0();
const LaunchTable &launch_table_16_2_1();
const LaunchTable &launch_table_16_4_0();
const LaunchTable &launch_table_16_4_1();
const LaunchTable &launch_table_17_3_0();
const LaunchTable &launch_table_17_3_1();
const LaunchTable &launch_table_17_2_0();
const LaunchTable &launch_table_17_2_1();
const LaunchTable &launch_table_17_4_0();
const LaunchTable &launch_table_17_4_1();

namespace {
// [log N][radix log 2..4][column tile 0/1]; sizes with one pass (N <= 2^12) have no
// column pass, so both column-tile entries name the same launchers.
using TableFn = const LaunchTable &(*)();
struct TableSet {
  TableFn fn[18][5][2] = {};
  TableSet() {
#define KS_T0(N)                                \
  for (int c = 0; c < 2; ++c) {                 \
    fn[N][3][c] = &launch_table_##N##_3_0;      \
    fn[N][2][c] = &launch_table_##N##_2_0;      \
    fn[N][4][c] = &launch_table_##N##_4_0;      \
  }
#define KS_T1(N)                            \
  fn[N][3][0] = &launch_table_##N##_3_0;    \
  fn[N][2][0] = &launch_table_##N##_2_0;    \
  fn[N][4][0] = &launch_table_##N##_4_0;    \
  fn[N][3][1] = &launch_table_##N##_3_1;    \
  fn[N][2][1] = &launch_table_##N##_2_1;    \
  fn[N][4][1] = &launch_table_##N##_4_1;
    KS_T0(1) KS_T0(2) KS_T0(3) KS_T0(4) KS_T0(5) KS_T0(6) KS_T0(7) KS_T0(8) KS_T0(9)
    KS_T0(10) KS_T0(11) KS_T0(12)
    KS_T1(13) KS_T1(14) KS_T1(15) KS_T1(16) KS_T1(17)
#undef KS_T0
#undef KS_T1
  }
};
}  // namespace

const LaunchTable *launch_table(int logn, int rl, int ca) {
  static const TableSet t;
  if (logn < 1 || logn > 17 || rl < 2 || rl > 4 || ca < 0 || ca > 1) return nullptr;
  const TableFn f = t.fn[logn][rl][ca];
  return f ? &f() : nullptr;
}

namespace kern {
cudaError_t smem_opt_in(const void *kernel, int bytes) {
  static std::mutex mu;
  static std::unordered_map<const void *, cudaError_t> done;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find(kernel);
  if (it != done.end()) return it->second;
  cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  done[kernel] = r;
  return r;
}
}  // namespace kern
}  // namespace ks
