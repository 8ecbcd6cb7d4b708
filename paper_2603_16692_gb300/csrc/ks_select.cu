// The learned dataflow selector inside the library (the parameter-aware choice of
// dataflow that Sec. V proposes): an installed 6-64-64-4 network (parameters trained
// by ks_mlp_train) picks a context's plan with one ks_mlp_forward launch.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "ks_internal.h"

namespace {

struct SelectorState {
  std::mutex mu;
  bool loaded = false;
  ks_selector sel;
  float *dev = nullptr;  // parameters, then the feature row, then the outputs
  int device = -1;
  unsigned gen = 0;      // bumped by every ks_selector_load
};
SelectorState g_sel;

// Offsets (floats) of the feature row and the outputs in the device buffer; both are
// 16-byte aligned (KS_MLP_PARAMS is a multiple of 4).
constexpr int kX = KS_MLP_PARAMS, kY = KS_MLP_PARAMS + 8, kFloats = KS_MLP_PARAMS + 16;
static_assert(KS_MLP_PARAMS % 4 == 0, "aligned feature row");

bool plan_ok(int v, int ch) {
  const int base = v & 0xff;
  if (base < KS_DSOB || base > KS_DPOC) return false;
  if (v & ~(0xff | KS_UNFUSED | KS_RADIX4 | KS_RADIX16)) return false;
  if ((v & KS_RADIX4) && (v & KS_RADIX16)) return false;
  return ch >= 0 && ch <= 64;
}

}  // namespace

extern "C" {

int ks_selector_load(const ks_selector *sel) {
  if (!sel || sel->l2_bytes < 0) return KS_EINVAL;
  for (int k = 0; k < 6; ++k)
    if (!(sel->x_std[k] > 0) || !std::isfinite(sel->x_mean[k]) || !std::isfinite(sel->x_std[k]))
      return KS_EINVAL;
  for (int k = 0; k < 4; ++k) {
    if (!(sel->t_std[k] > 0) || !std::isfinite(sel->t_mean[k]) || !std::isfinite(sel->t_std[k]))
      return KS_EINVAL;
    if (!plan_ok(sel->variant[k], sel->chunks[k])) return KS_EINVAL;
  }
  for (int k = 0; k < KS_MLP_PARAMS; ++k)
    if (!std::isfinite(sel->params[k])) return KS_EINVAL;
  std::lock_guard<std::mutex> lk(g_sel.mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return KS_ECUDA;
  }
  if (g_sel.dev && g_sel.device != dev) {
    // parameters of another device: free them there
    cudaSetDevice(g_sel.device);
    cudaFree(g_sel.dev);
    cudaSetDevice(dev);
    g_sel.dev = nullptr;
  }
  if (!g_sel.dev) {
    if (cudaMalloc(&g_sel.dev, kFloats * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      g_sel.dev = nullptr;
      g_sel.loaded = false;
      return KS_ENOMEM;
    }
    g_sel.device = dev;
  }
  // synchronous: the device's earlier work with the old parameters has finished
  if (cudaMemcpy(g_sel.dev, sel->params, KS_MLP_PARAMS * sizeof(float),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    g_sel.loaded = false;
    return KS_ECUDA;
  }
  g_sel.sel = *sel;
  g_sel.loaded = true;
  ++g_sel.gen;
  return KS_OK;
}

int ks_select(ks_context *c, int *variant, int *chunks, void *stream) {
  if (!c) return KS_EINVAL;
  std::lock_guard<std::mutex> lk(g_sel.mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return KS_ECUDA;
  }
  if (!g_sel.loaded || dev != g_sel.device) return KS_EINVAL;
  const ks_selector &S = g_sel.sel;
  double l2 = (double)S.l2_bytes;
  if (l2 <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      return KS_ECUDA;
    }
    l2 = v;
  }
  // features: log2 N, L+1, dnum (the digit count for a level view), and the ModUp
  // working sets of DPOB and DSOB and the key bytes against L2 (log2)
  const double n8 = (double)c->N * 8, qp = c->qp, beta = c->beta;
  const double f[6] = {(double)c->logn,
                       (double)c->nq,
                       (double)(c->top_L >= 0 ? c->beta : c->dnum),
                       std::log2(beta * qp * n8 / l2),
                       std::log2(qp * n8 / l2),
                       std::log2(2 * beta * qp * n8 / l2)};
  float x[6];
  for (int k = 0; k < 6; ++k) x[k] = (float)((f[k] - S.x_mean[k]) / S.x_std[k]);
  cudaStream_t s = (cudaStream_t)stream;
  float y[4];
  if (cudaMemcpyAsync(g_sel.dev + kX, x, sizeof(x), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return KS_ECUDA;
  }
  const int rc = ks_mlp_forward(g_sel.dev, g_sel.dev + kX, 1, g_sel.dev + kY, stream);
  if (rc) return rc;
  if (cudaMemcpyAsync(y, g_sel.dev + kY, sizeof(y), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return KS_ECUDA;
  }
  // outputs: standardised [log t_0, log t_k - log t_0]; pick the smallest log t_k
  const double e0 = y[0] * S.t_std[0] + S.t_mean[0];
  int best = 0;
  double lbest = e0;
  for (int k = 1; k < 4; ++k) {
    const double lk_ = e0 + (y[k] * S.t_std[k] + S.t_mean[k]);
    if (lk_ < lbest) {
      lbest = lk_;
      best = k;
    }
  }
  c->sel_variant = S.variant[best];
  c->sel_chunks = S.chunks[best];
  c->sel_gen = g_sel.gen;
  if (variant) *variant = c->sel_variant;
  if (chunks) *chunks = c->sel_chunks;
  return KS_OK;
}

}  // extern "C"

namespace ks {

bool selected_current(const ks_context *c) {
  std::lock_guard<std::mutex> lk(g_sel.mu);
  return c && g_sel.loaded && c->sel_variant > 0 && c->sel_gen == g_sel.gen;
}

}  // namespace ks
