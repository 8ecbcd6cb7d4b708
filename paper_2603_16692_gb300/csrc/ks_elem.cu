// Element-wise KeySwitch kernels (sm_103a): the unfused building blocks
// (BConv, key multiply, ModDown scaling as separate passes) and the key-generation
// helpers. Coalesced one-word-per-thread loops; grid (blocks over N, tasks).
#include <cuda_runtime.h>

#include "ks_arith.cuh"
#include "ks_internal.h"
#include "ks_kern.cuh"

namespace ks {
namespace {

using EArgs = kern::KArgs;
inline EArgs eargs(const ks_context *c) { return kern::make_args(c); }
using kern::decode;

// y = sum_k src_k[n] * cst[k] reduced by REDC in runs of `run` terms, canonical.
__device__ __forceinline__ u64 bconv_point(const u64 *__restrict__ src, size_t N, size_t n,
                                           int ns, const u64 *cst, int run, const ModInfo &mi) {
  u64 z = 0;
  int k = 0;
  while (k < ns) {
    const int kend = min(ns, k + run);
    U128 acc = {0, 0};
    for (; k < kend; ++k) mac128(acc, __ldg(src + (size_t)k * N + n), cst[k]);
    z = csub(z + csub(redc(acc, mi.m, mi.minv), mi.m), mi.m);
  }
  return z;
}

// ModUp BConv of digit j onto limb t (Montgomery-scaled), TASK_UP item (t, j, slot).
__global__ void k_bconv_up(EArgs a, JobSet js, WsOff wo, Tasks tk) {
  pdl_wait();
  __shared__ u64 cst[kMaxLimbs];
  const JobPtr jp = js.j[blockIdx.z];
  const u64 *v = jp.ws + wo.v;
  u64 *tmp = jp.ws + wo.tmp;
  const uint32_t w = decode(a, tk, blockIdx.y);
  const int t = task_limb(w), j = task_dig(w);
  const int i0 = j * a.alpha, ns = min(a.nq, i0 + a.alpha) - i0;
  for (int k = threadIdx.x; k < ns; k += blockDim.x)
    cst[k] = a.tab.cup[((size_t)j * a.qp + t) * a.alpha + k];
  __syncthreads();
  const ModInfo mi = a.tab.mod[t];
  const size_t N = a.N;
  u64 *o = tmp + (size_t)task_slot(w) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x)
    o[n] = bconv_point(v + (size_t)i0 * N, N, n, ns, cst, a.run_up, mi);
  pdl_trigger();
}

// ModDown BConv of the P-limbs of polynomial c onto q_i, TASK_DOWN item (i, c, slot).
__global__ void k_bconv_down(EArgs a, JobSet js, WsOff wo, Tasks tk) {
  pdl_wait();
  __shared__ u64 cst[kMaxLimbs];
  const JobPtr jp = js.j[blockIdx.z];
  const u64 *vp = jp.ws + wo.vp;
  u64 *tmp2 = jp.ws + wo.tmp2;
  const uint32_t w = decode(a, tk, blockIdx.y);
  const int i = task_limb(w), c = task_dig(w);
  for (int k = threadIdx.x; k < a.np; k += blockDim.x)
    cst[k] = a.tab.cdown[(size_t)i * a.alpha + k];
  __syncthreads();
  const ModInfo mi = a.tab.mod[i];
  const size_t N = a.N;
  u64 *o = tmp2 + (size_t)task_slot(w) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x)
    o[n] = bconv_point(vp + (size_t)c * a.np * N, N, n, a.np, cst, a.run_down, mi);
  pdl_trigger();
}

// acc_c[t] (+)= sum_{j0 <= j < j1} ext_j[t] * evk[j][c][t], TASK_TARGET item t.
__global__ void k_keymult(EArgs a, JobSet js, WsOff wo, Tasks tk) {
  pdl_wait();
  const JobPtr jp = js.j[blockIdx.z];
  const u64 *tmp = jp.ws + wo.tmp;
  u64 *acc = jp.ws + wo.acc;
  const int t = task_limb(decode(a, tk, blockIdx.y));
  const ModInfo mi = a.tab.mod[t];
  const size_t N = a.N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    U128 s0 = {0, 0}, s1 = {0, 0};
    for (int j = tk.j0; j < tk.j1; ++j) {
      const int lo = j * a.alpha, hi = min(lo + a.alpha, a.nq);
      u64 y;
      if (t >= lo && t < hi)
        y = csub(shoup(__ldg(jp.d + (size_t)t * N + n), mi.r1, mi.r1s, mi.m), mi.m);
      else
        y = __ldg(tmp + (size_t)(j * tk.sm.sj + t * tk.sm.st + tk.sm.base) * N + n);
      mac128(s0, y, __ldg(jp.evk + kern::evk_off(a, j, 0, t) + n));
      mac128(s1, y, __ldg(jp.evk + kern::evk_off(a, j, 1, t) + n));
    }
    u64 r0v = csub(redc(s0, mi.m, mi.minv), mi.m);
    u64 r1v = csub(redc(s1, mi.m, mi.minv), mi.m);
    u64 *a0 = acc + (size_t)t * N + n;
    u64 *a1 = acc + ((size_t)a.qp + t) * N + n;
    if (!tk.first) {
      r0v = addmod(r0v, *a0, mi.m);
      r1v = addmod(r1v, *a1, mi.m);
    }
    *a0 = r0v;
    *a1 = r1v;
  }
  pdl_trigger();
}

// out_c[i] = (acc_c[i] - zhat) * P^-1, TASK_DOWN item (i, c, slot of zhat).
__global__ void k_moddown_scale(EArgs a, JobSet js, WsOff wo, Tasks tk) {
  pdl_wait();
  const JobPtr jp = js.j[blockIdx.z];
  const uint32_t w = decode(a, tk, blockIdx.y);
  const int i = task_limb(w), c = task_dig(w);
  const u64 m = a.tab.mod[i].m;
  const ulonglong2 pv = a.tab.pinv[i];
  const size_t N = a.N;
  const u64 *z = jp.ws + wo.tmp2 + (size_t)task_slot(w) * N;
  const u64 *ac = jp.ws + wo.acc + ((size_t)c * a.qp + i) * N;
  const size_t ob = ((size_t)c * a.nq + i) * N;
  u64 *o = jp.out + ob;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x)
    o[n] = kern::out_word(jp, c, ob + n,
                          csub(shoup(__ldg(ac + n) + m - __ldg(z + n), pv.x, pv.y, m), m), m);
  pdl_trigger();
}

// polys [2 + beta][QP][N]: 0 = s_from, 1 = s_to, 2 + j = e_j, as residues mod each prime.
// With kinv != 0, s_from is replaced by sigma_k(s_from)(x) = s_from(x^k): output
// coefficient n takes source n1 = n k^-1 mod 2N, negated when n1 >= N (x^N = -1).
__global__ void k_keygen_lift(EArgs a, const int8_t *__restrict__ sf,
                              const int8_t *__restrict__ st, const int32_t *__restrict__ e,
                              unsigned kinv, u64 *polys) {
  const int poly = blockIdx.z, t = blockIdx.y;
  const u64 m = a.tab.mod[t].m;
  const size_t N = a.N;
  u64 *o = polys + ((size_t)poly * a.qp + t) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    long long x;
    if (poly == 0 && kinv) {
      const size_t n1 = (n * kinv) & (2 * N - 1);
      x = n1 < N ? sf[n1] : -(long long)sf[n1 - N];
    } else if (poly == 0)
      x = sf[n];
    else if (poly == 1)
      x = st[n];
    else
      x = e[(size_t)(poly - 2) * N + n];
    const u64 r = (u64)(x < 0 ? -x : x) % m;
    o[n] = (x < 0 && r) ? m - r : r;
  }
}

// x*y mod m for arbitrary canonical x, y: two Montgomery reductions (x y 2^-64, then * 2^128).
__device__ __forceinline__ u64 mulmod_full(u64 x, u64 y, const ModInfo &mi) {
  U128 p = {0, 0};
  mac128(p, x, y);
  const u64 t = csub(redc(p, mi.m, mi.minv), mi.m);
  U128 p2 = {0, 0};
  mac128(p2, t, mi.r2);
  return csub(redc(p2, mi.m, mi.minv), mi.m);
}

// evk[j][0][t] = -a_j s_to + e_j + [P g_j]_t s_from; evk[j][1][t] = a_j.
__global__ void k_keygen_combine(EArgs a, const u64 *__restrict__ polys,
                                 const u64 *__restrict__ arand, u64 *evk) {
  const int j = blockIdx.z, t = blockIdx.y;
  const ModInfo mi = a.tab.mod[t];
  const u64 m = mi.m;
  const size_t N = a.N;
  const bool in_digit = t < a.nq && t >= j * a.alpha && t < min((j + 1) * a.alpha, a.nq);
  const u64 pg = in_digit ? a.tab.pmod[t].x : 0;
  const u64 *sf = polys + ((size_t)0 * a.qp + t) * N;
  const u64 *st = polys + ((size_t)1 * a.qp + t) * N;
  const u64 *ej = polys + ((size_t)(2 + j) * a.qp + t) * N;
  const u64 *aj = arand + ((size_t)j * a.qp + t) * N;
  u64 *b = evk + ((size_t)(j * 2 + 0) * a.qp + t) * N;
  u64 *ao = evk + ((size_t)(j * 2 + 1) * a.qp + t) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    const u64 av = aj[n];
    u64 v = ej[n];
    const u64 as = mulmod_full(av, st[n], mi);
    v = v >= as ? v - as : v + m - as;
    v = addmod(v, mulmod_full(pg, sf[n], mi), m);
    b[n] = v;
    ao[n] = av;
  }
}

__global__ void k_keygen_square(EArgs a, u64 *polys) {
  const int t = blockIdx.y;
  const ModInfo mi = a.tab.mod[t];
  const size_t N = a.N;
  u64 *o = polys + (size_t)t * N;  // poly 0 = s_from
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x)
    o[n] = mulmod_full(o[n], o[n], mi);
}

// x*y + z*w mod m for canonical inputs: the exact 128-bit sum (< 2 m^2 < m 2^64) is
// reduced once, then the 2^-64 of REDC is undone by a second REDC against 2^128 mod m.
__device__ __forceinline__ u64 mulmod2_full(u64 x, u64 y, u64 z, u64 w, const ModInfo &mi) {
  U128 p = {0, 0};
  mac128(p, x, y);
  mac128(p, z, w);
  const u64 t = csub(redc(p, mi.m, mi.minv), mi.m);
  U128 p2 = {0, 0};
  mac128(p2, t, mi.r2);
  return csub(redc(p2, mi.m, mi.minv), mi.m);
}

// HMUL tensor product, limb i = blockIdx.y. Each thread reads its four words before
// it writes, so out may alias x or y.
__global__ void k_tensor(EArgs a, const u64 *x, const u64 *y, u64 *out, u64 *d2) {
  pdl_wait();
  const int i = blockIdx.y;
  const ModInfo mi = a.tab.mod[i];
  const size_t N = a.N, P = (size_t)a.nq * N, off = (size_t)i * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    const u64 x0 = x[off + n], x1 = x[P + off + n], y0 = y[off + n], y1 = y[P + off + n];
    const u64 r0 = mulmod_full(x0, y0, mi);
    const u64 r1 = mulmod2_full(x0, y1, x1, y0, mi);
    const u64 r2 = mulmod_full(x1, y1, mi);
    out[off + n] = r0;
    out[P + off + n] = r1;
    d2[off + n] = r2;
  }
  pdl_trigger();
}

// Galois automorphism in the NTT domain. Slot j holds a(w_j), w_j = psi^(2 brv(j) + 1);
// sigma_k(a)(w_j) = a(w_j^k) = a(w_j') with 2 brv(j') + 1 = (2 brv(j) + 1) k mod 2N,
// so the automorphism is the gather y[j] = x[j']. Limb i = blockIdx.y, c = blockIdx.z.
__global__ void k_automorph(EArgs a, int logn, const u64 *__restrict__ ct, unsigned k,
                            u64 *y0, u64 *y1) {
  pdl_wait();
  const int i = blockIdx.y, c = blockIdx.z;
  const size_t N = a.N;
  const u64 *x = ct + ((size_t)c * a.nq + i) * N;
  u64 *y = (c == 0 ? y0 : y1) + (size_t)i * N;
  const unsigned mask2n = (unsigned)(2 * N - 1), sh = 32 - logn;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    const unsigned e = (2u * (__brev((unsigned)n) >> sh) + 1u) * k & mask2n;
    const unsigned src = __brev((e - 1u) >> 1) >> sh;
    y[n] = __ldg(x + src);
  }
  pdl_trigger();
}

int ew_blocks(size_t N) {
  const size_t b = (N + 1023) / 1024;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_bconv_up(const ks_context *c, const JobSet &js, const WsOff &o,
                            const Tasks &tk, int count, cudaStream_t s) {
  if (count == 0 || js.n == 0) return cudaSuccess;
  return launch_pdl(k_bconv_up, dim3(ew_blocks(c->N), count, js.n), dim3(256), 0, s, eargs(c),
                    js, o, tk);
}

cudaError_t launch_bconv_down(const ks_context *c, const JobSet &js, const WsOff &o,
                              const Tasks &tk, int count, cudaStream_t s) {
  if (count == 0 || js.n == 0) return cudaSuccess;
  return launch_pdl(k_bconv_down, dim3(ew_blocks(c->N), count, js.n), dim3(256), 0, s, eargs(c),
                    js, o, tk);
}

cudaError_t launch_keymult(const ks_context *c, const JobSet &js, const WsOff &o,
                           const Tasks &tk, cudaStream_t s) {
  const int count = tk.t1 - tk.t0;
  if (count <= 0 || js.n == 0) return cudaSuccess;
  return launch_pdl(k_keymult, dim3(ew_blocks(c->N), count, js.n), dim3(256), 0, s, eargs(c), js,
                    o, tk);
}

cudaError_t launch_moddown_scale(const ks_context *c, const JobSet &js, const WsOff &o,
                                 const Tasks &tk, int count, cudaStream_t s) {
  if (count == 0 || js.n == 0) return cudaSuccess;
  return launch_pdl(k_moddown_scale, dim3(ew_blocks(c->N), count, js.n), dim3(256), 0, s,
                    eargs(c), js, o, tk);
}

cudaError_t launch_keygen_lift(const ks_context *c, const int8_t *sf, const int8_t *st,
                               const int32_t *e, unsigned kinv, u64 *polys, cudaStream_t s) {
  k_keygen_lift<<<dim3(ew_blocks(c->N), c->qp, 2 + c->beta), 256, 0, s>>>(eargs(c), sf, st, e,
                                                                          kinv, polys);
  return cudaGetLastError();
}

cudaError_t launch_keygen_square(const ks_context *c, u64 *polys, cudaStream_t s) {
  k_keygen_square<<<dim3(ew_blocks(c->N), c->qp), 256, 0, s>>>(eargs(c), polys);
  return cudaGetLastError();
}

cudaError_t launch_tensor(const ks_context *c, const u64 *x, const u64 *y, u64 *out, u64 *d2,
                          cudaStream_t s) {
  return launch_pdl(k_tensor, dim3(ew_blocks(c->N), c->nq), dim3(256), 0, s, eargs(c), x, y, out,
                    d2);
}

cudaError_t launch_automorph(const ks_context *c, const u64 *ct, unsigned k, u64 *y0, u64 *y1,
                             cudaStream_t s) {
  return launch_pdl(k_automorph, dim3(ew_blocks(c->N), c->nq, 2), dim3(256), 0, s, eargs(c),
                    c->logn, ct, k, y0, y1);
}

cudaError_t launch_keygen_combine(const ks_context *c, const u64 *polys, const u64 *arand,
                                  u64 *evk, cudaStream_t s) {
  k_keygen_combine<<<dim3(ew_blocks(c->N), c->qp, c->beta), 256, 0, s>>>(eargs(c), polys, arand,
                                                                        evk);
  return cudaGetLastError();
}

}  // namespace ks
