// Dataflow-selector MLP (6 -> 64 -> 64 -> 4, ReLU, FP32): inference, gradients and
// full-batch Adam training as hand-written CUDA kernels. The network predicts the
// (normalised) log-latency of the four dataflows from workload features; it never
// touches the KeySwitch arithmetic.
//
// Parameters are one float array (KS_MLP_PARAMS floats):
//   W1 [6][64] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64][4] | b3 [4]
// with W[i][j] the weight from input i to output j.
//
// Training runs in one CTA over the whole batch (B <= KS_MLP_MAX_BATCH rows): forward,
// masked mean-squared loss, backward and the Adam update, `steps` times in one
// launch. The rows pass through shared memory in chunks of CH; every gradient entry
// is summed by one thread, chunk after chunk in row order, so results are
// deterministic and equal to the full-batch gradient.
#include <cuda_runtime.h>

#include "ks_internal.h"

namespace {

constexpr int IN = 6, H = 64, OUT = 4;
constexpr int OW1 = 0, OB1 = OW1 + IN * H, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + H * OUT, NP = OB3 + OUT;
constexpr int NT = 256;
constexpr int CH = 256;  // rows per chunk held in shared memory

static_assert(NP == KS_MLP_PARAMS, "parameter layout");

struct Smem {
  float *p, *x, *h1, *h2, *y, *dh;
};

__device__ Smem carve(float *s, int B) {
  Smem m;
  m.p = s;
  m.x = m.p + NP;
  m.h1 = m.x + B * IN;
  m.h2 = m.h1 + B * H;
  m.y = m.h2 + B * H;
  m.dh = m.y + B * OUT;
  return m;
}

__host__ __device__ constexpr size_t smem_floats(int B) {
  return (size_t)NP + (size_t)B * (IN + H + H + OUT + H);
}

__device__ void forward(const Smem &m, int B) {
  for (int k = threadIdx.x; k < B * H; k += NT) {
    const int b = k / H, j = k % H;
    float a = m.p[OB1 + j];
#pragma unroll
    for (int i = 0; i < IN; ++i) a += m.x[b * IN + i] * m.p[OW1 + i * H + j];
    m.h1[k] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < B * H; k += NT) {
    const int b = k / H, j = k % H;
    float a = m.p[OB2 + j];
    for (int i = 0; i < H; ++i) a += m.h1[b * H + i] * m.p[OW2 + i * H + j];
    m.h2[k] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < B * OUT; k += NT) {
    const int b = k / OUT, o = k % OUT;
    float a = m.p[OB3 + o];
    for (int i = 0; i < H; ++i) a += m.h2[b * H + i] * m.p[OW3 + i * OUT + o];
    m.y[k] = a;
  }
  __syncthreads();
}

// Masked squared error of a chunk, sum mask (y - t)^2 / total, and its gradient
// added into g (written when first): leaves dL/dy in m.y. Returns the chunk's loss part.
__device__ float backward(const Smem &m, int B, const float *t, const float *mask, float total,
                          bool first, float *g, float *red) {
  float loss = 0.f;
  for (int k = threadIdx.x; k < B * OUT; k += NT) {
    const float d = m.y[k] - t[k];
    loss += mask[k] * d * d;
  }
  red[threadIdx.x] = loss;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const float L = red[0] / total;
  __syncthreads();
  for (int k = threadIdx.x; k < B * OUT; k += NT) m.y[k] = mask[k] * 2.f * (m.y[k] - t[k]) / total;
  __syncthreads();
  // layer 3: dW3 = h2^T dy, db3 = sum dy
  for (int k = threadIdx.x; k < H * OUT + OUT; k += NT) {
    float a = 0.f;
    if (k < H * OUT) {
      const int i = k / OUT, o = k % OUT;
      for (int b = 0; b < B; ++b) a += m.h2[b * H + i] * m.y[b * OUT + o];
      g[OW3 + k] = first ? a : g[OW3 + k] + a;
    } else {
      const int o = k - H * OUT;
      for (int b = 0; b < B; ++b) a += m.y[b * OUT + o];
      g[OB3 + o] = first ? a : g[OB3 + o] + a;
    }
  }
  // dh2 = (dy W3^T) * [h2 > 0]
  for (int k = threadIdx.x; k < B * H; k += NT) {
    const int b = k / H, i = k % H;
    float a = 0.f;
#pragma unroll
    for (int o = 0; o < OUT; ++o) a += m.y[b * OUT + o] * m.p[OW3 + i * OUT + o];
    m.dh[k] = m.h2[k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // layer 2: dW2 = h1^T dh2, db2 = sum dh2
  for (int k = threadIdx.x; k < H * H + H; k += NT) {
    float a = 0.f;
    if (k < H * H) {
      const int i = k / H, j = k % H;
      for (int b = 0; b < B; ++b) a += m.h1[b * H + i] * m.dh[b * H + j];
      g[OW2 + k] = first ? a : g[OW2 + k] + a;
    } else {
      const int j = k - H * H;
      for (int b = 0; b < B; ++b) a += m.dh[b * H + j];
      g[OB2 + j] = first ? a : g[OB2 + j] + a;
    }
  }
  // dh1 = (dh2 W2^T) * [h1 > 0], written over h2 (no longer needed)
  for (int k = threadIdx.x; k < B * H; k += NT) {
    const int b = k / H, i = k % H;
    float a = 0.f;
    for (int j = 0; j < H; ++j) a += m.dh[b * H + j] * m.p[OW2 + i * H + j];
    m.h2[k] = m.h1[k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // layer 1: dW1 = x^T dh1, db1 = sum dh1
  for (int k = threadIdx.x; k < IN * H + H; k += NT) {
    float a = 0.f;
    if (k < IN * H) {
      const int i = k / H, j = k % H;
      for (int b = 0; b < B; ++b) a += m.x[b * IN + i] * m.h2[b * H + j];
      g[OW1 + k] = first ? a : g[OW1 + k] + a;
    } else {
      const int j = k - IN * H;
      for (int b = 0; b < B; ++b) a += m.h2[b * H + j];
      g[OB1 + j] = first ? a : g[OB1 + j] + a;
    }
  }
  __syncthreads();
  return L;
}

// Sum of the mask over all rows (the loss denominator; 1 if the mask is empty).
__device__ float mask_total(const float *mask, int B, float *red) {
  float cnt = 0.f;
  for (int k = threadIdx.x; k < B * OUT; k += NT) cnt += mask[k];
  red[threadIdx.x] = cnt;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const float total = red[0] > 0.f ? red[0] : 1.f;
  __syncthreads();
  return total;
}

// Loss and full-batch gradient (into g) over all B rows, chunk by chunk.
__device__ float loss_grad(const Smem &m, const float *x, const float *t, const float *mask,
                           int B, float total, float *g, float *red) {
  float L = 0.f;
  for (int r0 = 0; r0 < B; r0 += CH) {
    const int nb = min(CH, B - r0);
    for (int k = threadIdx.x; k < nb * IN; k += NT) m.x[k] = x[(size_t)r0 * IN + k];
    __syncthreads();
    forward(m, nb);
    L += backward(m, nb, t + (size_t)r0 * OUT, mask + (size_t)r0 * OUT, total, r0 == 0, g, red);
  }
  return L;
}

__device__ void load_params(const Smem &m, const float *params) {
  for (int k = threadIdx.x; k < NP; k += NT) m.p[k] = params[k];
  __syncthreads();
}

__global__ void __launch_bounds__(NT) k_mlp_forward(const float *params, const float *x, int B,
                                                    float *y) {
  extern __shared__ float s[];
  const Smem m = carve(s, CH);
  load_params(m, params);
  for (int r0 = 0; r0 < B; r0 += CH) {
    const int nb = min(CH, B - r0);
    for (int k = threadIdx.x; k < nb * IN; k += NT) m.x[k] = x[(size_t)r0 * IN + k];
    __syncthreads();
    forward(m, nb);
    for (int k = threadIdx.x; k < nb * OUT; k += NT) y[(size_t)r0 * OUT + k] = m.y[k];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(NT) k_mlp_grad(const float *params, const float *x,
                                                 const float *t, const float *mask, int B,
                                                 float *grad, float *loss) {
  extern __shared__ float s[];
  __shared__ float red[NT];
  const Smem m = carve(s, CH);
  load_params(m, params);
  const float total = mask_total(mask, B, red);
  const float L = loss_grad(m, x, t, mask, B, total, grad, red);
  if (threadIdx.x == 0) *loss = L;
}

// `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8); the loss of every
// step goes to loss[step].
__global__ void __launch_bounds__(NT) k_mlp_train(float *params, float *adam_m, float *adam_v,
                                                  float *grad, const float *x, const float *t,
                                                  const float *mask, int B, int steps, float lr,
                                                  int step0, float *loss) {
  extern __shared__ float s[];
  __shared__ float red[NT];
  const Smem m = carve(s, CH);
  load_params(m, params);
  const float total = mask_total(mask, B, red);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < steps; ++it) {
    const float L = loss_grad(m, x, t, mask, B, total, grad, red);
    if (threadIdx.x == 0) loss[it] = L;
    __syncthreads();  // the gradient is complete before the update reads it
    const int st = step0 + it + 1;
    const float c1 = 1.f - powf(b1, (float)st), c2 = 1.f - powf(b2, (float)st);
    for (int k = threadIdx.x; k < NP; k += NT) {
      const float gk = grad[k];
      const float mk = b1 * adam_m[k] + (1.f - b1) * gk;
      const float vk = b2 * adam_v[k] + (1.f - b2) * gk * gk;
      adam_m[k] = mk;
      adam_v[k] = vk;
      m.p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < NP; k += NT) params[k] = m.p[k];
}

int launch_check(size_t smem) {
  if (smem > 227 * 1024) return KS_EINVAL;
  return KS_OK;
}

int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return KS_OK;
  cudaGetLastError();
  return KS_ECUDA;
}

template <class K>
cudaError_t opt_in(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

extern "C" {

int ks_mlp_forward(const float *params, const float *x, int batch, float *y, void *stream) {
  if (!params || !x || !y || batch < 1 || batch > KS_MLP_MAX_BATCH) return KS_EINVAL;
  const size_t smem = smem_floats(CH) * sizeof(float);
  if (launch_check(smem)) return KS_EINVAL;
  cudaError_t e = opt_in(k_mlp_forward, smem);
  if (e) return rc_of(e);
  k_mlp_forward<<<1, NT, smem, (cudaStream_t)stream>>>(params, x, batch, y);
  return rc_of(cudaGetLastError());
}

int ks_mlp_grad(const float *params, const float *x, const float *t, const float *mask,
                int batch, float *grad, float *loss, void *stream) {
  if (!params || !x || !t || !mask || !grad || !loss || batch < 1 ||
      batch > KS_MLP_MAX_BATCH)
    return KS_EINVAL;
  const size_t smem = smem_floats(CH) * sizeof(float);
  if (launch_check(smem)) return KS_EINVAL;
  cudaError_t e = opt_in(k_mlp_grad, smem);
  if (e) return rc_of(e);
  k_mlp_grad<<<1, NT, smem, (cudaStream_t)stream>>>(params, x, t, mask, batch, grad, loss);
  return rc_of(cudaGetLastError());
}

int ks_mlp_train(float *params, float *adam_m, float *adam_v, float *grad_scratch,
                 const float *x, const float *t, const float *mask, int batch, int steps,
                 float lr, int step0, float *loss, void *stream) {
  if (!params || !adam_m || !adam_v || !grad_scratch || !x || !t || !mask || !loss ||
      batch < 1 || batch > KS_MLP_MAX_BATCH || steps < 0 || step0 < 0)
    return KS_EINVAL;
  if (steps == 0) return KS_OK;
  const size_t smem = smem_floats(CH) * sizeof(float);
  if (launch_check(smem)) return KS_EINVAL;
  cudaError_t e = opt_in(k_mlp_train, smem);
  if (e) return rc_of(e);
  k_mlp_train<<<1, NT, smem, (cudaStream_t)stream>>>(params, adam_m, adam_v, grad_scratch, x, t,
                                                     mask, batch, steps, lr, step0, loss);
  return rc_of(cudaGetLastError());
}

}  // extern "C"
