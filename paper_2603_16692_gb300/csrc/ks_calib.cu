// Calibration kernels: the throughput ceiling of the library's own modular
// arithmetic on this GPU, measured with every SM busy and no memory traffic. They
// give a measured denominator for the integer-bound kernels beside the one derived
// from unit counts and clocks.
//   KS_CAL_BUTTERFLY: forward lazy butterflies with the approximate Shoup product
//                     (the NTT inner operation for moduli below 2^51).
//   KS_CAL_MAC:       exact 64x64->128-bit multiply-accumulates (the basis-conversion
//                     and key-multiply inner operation), one REDC per 8 terms.
#include <cuda_runtime.h>

#include <algorithm>

#include "ks_arith.cuh"
#include "ks_internal.h"

namespace ks {
namespace {

constexpr int kCalThreads = 256;
constexpr int kChains = 8;  // independent dependency chains per thread

__device__ __forceinline__ void bfly(u64 &a, u64 &b, u64 w, u64 wp, u64 m, u64 m4) {
  const u64 t = shoup4(b, w, wp, m);
  const u64 x = a;
  a = x + t;
  b = x - t + m4;
}

__global__ void __launch_bounds__(kCalThreads) k_cal_butterfly(u64 m, u64 w, u64 wp, int iters,
                                                               u64 *sink) {
  u64 a[kChains], b[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = (threadIdx.x * 7919ull + c * 104729ull + blockIdx.x) % m;
    b[c] = (threadIdx.x * 15485863ull + c * 32452843ull) % m;
  }
  const u64 m4 = 4 * m;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      bfly(a[c], b[c], w, wp, m, m4);
      // keep the values bounded like a transform does between stages
      a[c] = a[c] >= m4 ? a[c] - m4 : a[c];
    }
  }
  u64 acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= a[c] ^ b[c];
  if (acc == 0x5eed) sink[blockIdx.x] = acc;  // practically never: defeats elimination
}

__global__ void __launch_bounds__(kCalThreads) k_cal_mac(u64 m, u64 minv, u64 c0, int iters,
                                                         u64 *sink) {
  u64 x[kChains], z[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = (threadIdx.x * 7919ull + c * 104729ull + blockIdx.x) % m;
    z[c] = 0;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      U128 acc = {0, 0};
#pragma unroll
      for (int k = 0; k < 8; ++k) mac128(acc, x[c] + k, c0 + k);
      z[c] += redc(acc, m, minv);
      x[c] = z[c] & ((1ull << 49) - 1);
    }
  }
  u64 acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= z[c];
  if (acc == 0x5eed) sink[blockIdx.x] = acc;
}

}  // namespace
}  // namespace ks

extern "C" int ks_calibrate(int kind, int iters, double *ops_per_s, void *stream) {
  using namespace ks;
  if (!ops_per_s || iters < 1 || (kind != KS_CAL_BUTTERFLY && kind != KS_CAL_MAC))
    return KS_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
    cudaGetLastError();
    return KS_ECUDA;
  }
  cudaError_t e =
      kind == KS_CAL_BUTTERFLY
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cal_butterfly, kCalThreads, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cal_mac, kCalThreads, 0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return KS_ECUDA;
  }
  const int grid = sms * per_sm;
  cudaStream_t s = (cudaStream_t)stream;
  u64 *sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&sink, (size_t)grid * sizeof(u64)) || cudaEventCreate(&a) ||
      cudaEventCreate(&b)) {
    cudaGetLastError();
    if (sink) cudaFree(sink);
    if (a) cudaEventDestroy(a);
    return KS_ENOMEM;
  }
  // a 50-bit prime, a twiddle and its Shoup quotient floor(w 2^64 / m)
  const u64 m = 1125899906842177ull, w = 987654321987ull;
  const u64 wp = (u64)(((unsigned __int128)w << 64) / m);
  u64 minv = 1;  // -m^-1 mod 2^64 by Newton iteration
  for (int k = 0; k < 6; ++k) minv *= 2 - m * minv;
  minv = 0 - minv;
  auto launch = [&](int n) {
    if (kind == KS_CAL_BUTTERFLY)
      k_cal_butterfly<<<grid, kCalThreads, 0, s>>>(m, w, wp, n, sink);
    else
      k_cal_mac<<<grid, kCalThreads, 0, s>>>(m, minv, 0x123456789abull, n, sink);
  };
  launch(std::max(1, iters / 10));  // warm-up
  cudaEventRecord(a, s);
  launch(iters);
  cudaEventRecord(b, s);
  int rc = KS_OK;
  if (cudaEventSynchronize(b) != cudaSuccess) {
    rc = KS_ECUDA;
  } else {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double per_iter = kind == KS_CAL_BUTTERFLY ? kChains : 8.0 * kChains;
    *ops_per_s = (double)grid * kCalThreads * iters * per_iter / (ms * 1e-3);
  }
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  return rc;
}
