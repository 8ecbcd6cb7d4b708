// ks_switch_noalloc: a KeySwitch whose scratch memory is a fixed, file-scope
// device array instead of memory the caller or the library allocates.
//
// Some callers cannot allocate device memory at the time they switch keys: callers
// held to a memory-pool or allocator budget that forbids new device allocations
// once the budget is reached, and real-time or embedded integrations that must not
// touch the allocator (whose calls can block and synchronize the device) after
// start-up. For them this entry point uses a static scratch of kScratchBytes, which
// every GPU that loads this module holds until the process exits, and only launches
// kernels: no graph cache, no context arena.
#include <cuda_runtime.h>

#include <mutex>

#include "ks_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)128 << 20;  // 128 MiB

// The scratch itself. In host code `g_ks_scratch` names a host-side stand-in,
// not a device address: only the address from cudaGetSymbolAddress may be
// handed to kernels.
__device__ __align__(256) unsigned long long g_ks_scratch[kScratchBytes / 8];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch on device `dev`, looked up once per device with that
// device current (the caller has checked that it is). The address is cached for the
// life of the process: a device reset (cudaDeviceReset) is not supported with this
// entry point.
int scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return KS_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ks_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return KS_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return KS_OK;
}

}  // namespace

extern "C" {

size_t ks_noalloc_scratch_bytes(void) { return kScratchBytes; }

int ks_switch_noalloc(ks_context *ctx, const uint64_t *d_dev, const uint64_t *evk_dev,
                      uint64_t *out_dev, int variant, int chunks, void *stream) {
  if (!ctx || !d_dev || !evk_dev || !out_dev) return KS_EINVAL;
  size_t need = 0;
  int rc = ks_workspace_size(ctx, variant, chunks, &need);
  if (rc) return rc;
  if (need > kScratchBytes) return KS_EINVAL;  // does not fit the static scratch
  // The scratch address belongs to the current device: it must be the context's.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return KS_ECUDA;
  }
  if (dev != ctx->device) return KS_EINVAL;
  void *scratch = nullptr;
  rc = scratch_address(dev, &scratch);
  if (rc) return rc;
  return ks::switch_launch_only(ctx, d_dev, evk_dev, out_dev, variant, chunks, scratch,
                                kScratchBytes, stream);
}

}  // extern "C"
