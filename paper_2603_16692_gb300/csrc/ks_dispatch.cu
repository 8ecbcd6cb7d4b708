// Run-time selection of the per-N kernel launchers.
#include <mutex>
#include <unordered_map>

#include "ks_internal.h"

namespace ks {
const LaunchTable &launch_table_1_3();
const LaunchTable &launch_table_1_2();
const LaunchTable &launch_table_1_4();
const LaunchTable &launch_table_2_3();
const LaunchTable &launch_table_2_2();
const LaunchTable &launch_table_2_4();
const LaunchTable &launch_table_3_3();
const LaunchTable &launch_table_3_2();
const LaunchTable &launch_table_3_4();
const LaunchTable &launch_table_4_3();
const LaunchTable &launch_table_4_2();
const LaunchTable &launch_table_4_4();
const LaunchTable &launch_table_5_3();
const LaunchTable &launch_table_5_2();
const LaunchTable &launch_table_5_4();
const LaunchTable &launch_table_6_3();
const LaunchTable &launch_table_6_2();
const LaunchTable &launch_table_6_4();
const LaunchTable &launch_table_7_3();
const LaunchTable &launch_table_7_2();
const LaunchTable &launch_table_7_4();
const LaunchTable &launch_table_8_3();
const LaunchTable &launch_table_8_2();
const LaunchTable &launch_table_8_4();
const LaunchTable &launch_table_9_3();
const LaunchTable &launch_table_9_2();
const LaunchTable &launch_table_9_4();
const LaunchTable &launch_table_10_3();
const LaunchTable &launch_table_10_2();
const LaunchTable &launch_table_10_4();
const LaunchTable &launch_table_11_3();
const LaunchTable &launch_table_11_2();
const LaunchTable &launch_table_11_4();
const LaunchTable &launch_table_12_3();
const LaunchTable &launch_table_12_2();
const LaunchTable &launch_table_12_4();
const LaunchTable &launch_table_13_3();
const LaunchTable &launch_table_13_2();
const LaunchTable &launch_table_13_4();
const LaunchTable &launch_table_14_3();
const LaunchTable &launch_table_14_2();
const LaunchTable &launch_table_14_4();
const LaunchTable &launch_table_15_3();
const LaunchTable &launch_table_15_2();
const LaunchTable &launch_table_15_4();
const LaunchTable &launch_table_16_3();
const LaunchTable &launch_table_16_2();
const LaunchTable &launch_table_16_4();
const LaunchTable &launch_table_17_3();
const LaunchTable &launch_table_17_2();
const LaunchTable &launch_table_17_4();

const LaunchTable *launch_table(int logn, int rl) {
  switch (rl == 4 ? logn * 4 + 4 + 128 : logn * 4 + rl) {
    case 7: return &launch_table_1_3();
    case 6: return &launch_table_1_2();
    case 136: return &launch_table_1_4();
    case 11: return &launch_table_2_3();
    case 10: return &launch_table_2_2();
    case 140: return &launch_table_2_4();
    case 15: return &launch_table_3_3();
    case 14: return &launch_table_3_2();
    case 144: return &launch_table_3_4();
    case 19: return &launch_table_4_3();
    case 18: return &launch_table_4_2();
    case 148: return &launch_table_4_4();
    case 23: return &launch_table_5_3();
    case 22: return &launch_table_5_2();
    case 152: return &launch_table_5_4();
    case 27: return &launch_table_6_3();
    case 26: return &launch_table_6_2();
    case 156: return &launch_table_6_4();
    case 31: return &launch_table_7_3();
    case 30: return &launch_table_7_2();
    case 160: return &launch_table_7_4();
    case 35: return &launch_table_8_3();
    case 34: return &launch_table_8_2();
    case 164: return &launch_table_8_4();
    case 39: return &launch_table_9_3();
    case 38: return &launch_table_9_2();
    case 168: return &launch_table_9_4();
    case 43: return &launch_table_10_3();
    case 42: return &launch_table_10_2();
    case 172: return &launch_table_10_4();
    case 47: return &launch_table_11_3();
    case 46: return &launch_table_11_2();
    case 176: return &launch_table_11_4();
    case 51: return &launch_table_12_3();
    case 50: return &launch_table_12_2();
    case 180: return &launch_table_12_4();
    case 55: return &launch_table_13_3();
    case 54: return &launch_table_13_2();
    case 184: return &launch_table_13_4();
    case 59: return &launch_table_14_3();
    case 58: return &launch_table_14_2();
    case 188: return &launch_table_14_4();
    case 63: return &launch_table_15_3();
    case 62: return &launch_table_15_2();
    case 192: return &launch_table_15_4();
    case 67: return &launch_table_16_3();
    case 66: return &launch_table_16_2();
    case 196: return &launch_table_16_4();
    case 71: return &launch_table_17_3();
    case 70: return &launch_table_17_2();
    case 200: return &launch_table_17_4();
    default: return nullptr;
  }
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
