// Run-time selection of the per-N kernel launchers.
#include <mutex>
#include <unordered_map>

#include "ks_internal.h"

namespace ks {
const LaunchTable &launch_table_1();
const LaunchTable &launch_table_2();
const LaunchTable &launch_table_3();
const LaunchTable &launch_table_4();
const LaunchTable &launch_table_5();
const LaunchTable &launch_table_6();
const LaunchTable &launch_table_7();
const LaunchTable &launch_table_8();
const LaunchTable &launch_table_9();
const LaunchTable &launch_table_10();
const LaunchTable &launch_table_11();
const LaunchTable &launch_table_12();
const LaunchTable &launch_table_13();
const LaunchTable &launch_table_14();
const LaunchTable &launch_table_15();
const LaunchTable &launch_table_16();
const LaunchTable &launch_table_17();

const LaunchTable *launch_table(int logn) {
  switch (logn) {
    case 1: return &launch_table_1();
    case 2: return &launch_table_2();
    case 3: return &launch_table_3();
    case 4: return &launch_table_4();
    case 5: return &launch_table_5();
    case 6: return &launch_table_6();
    case 7: return &launch_table_7();
    case 8: return &launch_table_8();
    case 9: return &launch_table_9();
    case 10: return &launch_table_10();
    case 11: return &launch_table_11();
    case 12: return &launch_table_12();
    case 13: return &launch_table_13();
    case 14: return &launch_table_14();
    case 15: return &launch_table_15();
    case 16: return &launch_table_16();
    case 17: return &launch_table_17();
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
