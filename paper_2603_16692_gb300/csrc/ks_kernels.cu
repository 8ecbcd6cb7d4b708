// KeySwitch kernels for sm_103a: two-pass negacyclic NTT / iNTT with the basis
// conversions fused into the first pass and the key multiply / ModDown scaling
// fused into the last pass (Sec. II-A, Fig. 1), plus the unfused building
// blocks and the key-generation helpers.
#include <cuda_runtime.h>

#include "ks_arith.cuh"
#include "ks_internal.h"
#include "ks_ntt.cuh"

namespace ks {

namespace {

constexpr int kEPT = 8;  // elements per thread in row-pass epilogues

enum { PRO_LOAD = 0, PRO_UP = 1, PRO_DOWN = 2 };

struct KArgs {
  Tables tab;
  Geo geo;
  int N, nq, np, qp, alpha, beta;
  int run_up, run_down;
};

KArgs make_args(const ks_context *c) {
  KArgs a;
  a.run_up = c->run_up;
  a.run_down = c->run_down;
  a.tab = c->tab;
  a.geo = c->geo;
  a.N = c->N;
  a.nq = c->nq;
  a.np = c->np;
  a.qp = c->qp;
  a.alpha = c->alpha;
  a.beta = c->beta;
  return a;
}

__device__ __forceinline__ int log2i(int x) { return 31 - __clz(x); }

__device__ __forceinline__ int pitch_of(int G) { return G == 1 ? 1 : G + 1; }

__device__ __forceinline__ TwAcc col_tw(const ulonglong2 *tab, int prime, int loga) {
  TwAcc t;
  t.tw = tab + ((size_t)prime << loga);
  t.off = 0;
  t.logstride = 0;
  t.rowbase = 0;
  t.rowstep = 0;
  return t;
}

__device__ __forceinline__ TwAcc row_tw(const ulonglong2 *tab, int prime, int loga, int logb,
                                        int r0) {
  TwAcc t;
  t.tw = tab + (size_t)prime * (((size_t)1 << logb) - 1) * ((size_t)1 << loga);
  t.off = 1;
  t.logstride = loga;
  t.rowbase = r0;
  t.rowstep = 1;
  return t;
}

// Row tile: element (x, g) <- src[(r0+g)*N2 + x], x fastest across threads.
// Plain (coherent) loads: some callers transform a buffer in place.
__device__ __forceinline__ void load_rows(u64 *s, const u64 *src, int logb, int logG, int P,
                                          int r0) {
  const int tile = 1 << (logb + logG);
  const int xm = (1 << logb) - 1;
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int g = e >> logb, x = e & xm;
    s[x * P + g] = src[((size_t)(r0 + g) << logb) + x];
  }
}

// Column tile: element (y, g) <- src[y*N2 + c0 + g], g fastest.
__device__ __forceinline__ void load_cols(u64 *s, const u64 *src, int loga, int logb,
                                          int logG, int P, int c0) {
  const int tile = 1 << (loga + logG);
  const int gm = (1 << logG) - 1;
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int y = e >> logG, g = e & gm;
    s[y * P + g] = src[((size_t)y << logb) + c0 + g];
  }
}

// Fast basis conversion into a tile: s[x*P+g] = REDC(sum_k src_k[gidx] * cst[k]).
// Element e -> (index into the limb, smem slot) by the tile geometry; `colmode`
// selects the column (g fastest) or row (x fastest) ordering. Sums are split in
// runs of at most `run` terms so that each stays below m 2^64.
__device__ __forceinline__ void bconv_tile(u64 *s, const u64 *__restrict__ src, size_t N,
                                           int nsrc, const u64 *cst, int run, bool colmode,
                                           int loga, int logb, int logG, int P, int base,
                                           u64 m, u64 minv) {
  const int logM = colmode ? loga : logb;
  const int tile = 1 << (logM + logG);
  const u64 m2 = 2 * m;
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    int x, g;
    size_t gidx;
    if (colmode) {
      x = e >> logG;
      g = e & ((1 << logG) - 1);
      gidx = ((size_t)x << logb) + base + g;
    } else {
      g = e >> logb;
      x = e & ((1 << logb) - 1);
      gidx = ((size_t)(base + g) << logb) + x;
    }
    u64 z = 0;
    int k = 0;
    while (k < nsrc) {
      const int kend = min(nsrc, k + run);
      U128 acc = {0, 0};
      for (; k < kend; ++k) mac128(acc, __ldg(src + (size_t)k * N + gidx), cst[k]);
      z += redc(acc, m, minv);
      z = z >= m2 ? z - m2 : z;
    }
    s[x * P + g] = z;
  }
}

// ---------------------------------------------------------------------------
// Inverse NTT, row pass (global stages logN-1 .. logN1). grid (N1/Gr, outer*inner).
// With a single pass (N1 == 1) it also applies the per-limb scale and writes
// canonical values.
__global__ void k_inv_row(KArgs a, const u64 *__restrict__ src, int src_outer, u64 *dst,
                          int dst_outer, int inner, int prime_base,
                          const ulonglong2 *__restrict__ scale) {
  extern __shared__ u64 sm[];
  const Geo &G = a.geo;
  const int logG = log2i(G.Gr), P = pitch_of(G.Gr);
  const int oi = blockIdx.y / inner, ii = blockIdx.y % inner;
  const int prime = prime_base + ii;
  const u64 m = a.tab.mod[prime].m;
  const size_t N = a.N;
  const u64 *s_l = src + ((size_t)oi * src_outer + ii) * N;
  u64 *d_l = dst + ((size_t)oi * dst_outer + ii) * N;
  const int r0 = blockIdx.x * G.Gr;
  load_rows(sm, s_l, G.logb, logG, P, r0);
  __syncthreads();
  tile_ntt_inv(sm, G.logb, logG, P, row_tw(a.tab.twr_i, prime, G.loga, G.logb, r0), m);
  const int tile = 1 << (G.logb + logG);
  const bool single = G.loga == 0;
  const ulonglong2 sc = scale[ii];
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int g = e >> G.logb, x = e & ((1 << G.logb) - 1);
    u64 v = sm[x * P + g];
    if (single) v = csub(shoup(v, sc.x, sc.y, m), m);
    d_l[((size_t)(r0 + g) << G.logb) + x] = v;
  }
}

// Inverse NTT, column pass (global stages logN1-1 .. 0) in place, then scale.
// grid (N2/Gc, outer*inner).
__global__ void k_inv_col(KArgs a, u64 *dst, int dst_outer, int inner, int prime_base,
                          const ulonglong2 *__restrict__ scale) {
  extern __shared__ u64 sm[];
  const Geo &G = a.geo;
  const int logG = log2i(G.Gc), P = pitch_of(G.Gc);
  const int oi = blockIdx.y / inner, ii = blockIdx.y % inner;
  const int prime = prime_base + ii;
  const u64 m = a.tab.mod[prime].m;
  u64 *d_l = dst + ((size_t)oi * dst_outer + ii) * (size_t)a.N;
  const int c0 = blockIdx.x * G.Gc;
  load_cols(sm, d_l, G.loga, G.logb, logG, P, c0);
  __syncthreads();
  tile_ntt_inv(sm, G.loga, logG, P, col_tw(a.tab.twc_i, prime, G.loga), m);
  const ulonglong2 sc = scale[ii];
  const int tile = 1 << (G.loga + logG);
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int y = e >> logG, g = e & ((1 << logG) - 1);
    d_l[((size_t)y << G.logb) + c0 + g] = csub(shoup(sm[y * P + g], sc.x, sc.y, m), m);
  }
}

// Stage the basis-conversion constants of one task into shared memory.
__device__ __forceinline__ void stage_consts(u64 *cst, const u64 *__restrict__ src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) cst[k] = __ldg(src + k);
}

// Produce a ModUp / ModDown / plain tile for task `w` (column or row mode).
// PRO_UP:   limb t = BConv of digit j's coefficient limbs (v) onto m_t,
//           Montgomery-scaled (constants carry 2^128).
// PRO_DOWN: limb i of polynomial c = BConv of the P-limbs vp[c] onto q_i.
// PRO_LOAD: the tile of buf[slot].
template <int PRO>
__device__ __forceinline__ void produce_tile(const KArgs &a, u64 *sm, u64 *cst, uint32_t w,
                                             const u64 *__restrict__ v, const u64 *buf,
                                             bool colmode, int logG, int P, int base) {
  const Geo &G = a.geo;
  const int t = task_limb(w);
  const size_t N = a.N;
  if (PRO == PRO_LOAD) {
    const u64 *b = buf + (size_t)task_slot(w) * N;
    if (colmode)
      load_cols(sm, b, G.loga, G.logb, logG, P, base);
    else
      load_rows(sm, b, G.logb, logG, P, base);
  } else if (PRO == PRO_UP) {
    const int j = task_dig(w);
    const int i0 = j * a.alpha;
    const int ns = min(a.nq, i0 + a.alpha) - i0;
    stage_consts(cst, a.tab.cup + ((size_t)j * a.qp + t) * a.alpha, ns);
    __syncthreads();
    const ModInfo mi = a.tab.mod[t];
    bconv_tile(sm, v + (size_t)i0 * N, N, ns, cst, a.run_up, colmode, G.loga, G.logb, logG, P,
               base, mi.m, mi.minv);
  } else {
    const int c = task_dig(w);
    stage_consts(cst, a.tab.cdown + (size_t)t * a.alpha, a.np);
    __syncthreads();
    const ModInfo mi = a.tab.mod[t];
    bconv_tile(sm, v + (size_t)c * a.np * N, N, a.np, cst, a.run_down, colmode, G.loga, G.logb,
               logG, P, base, mi.m, mi.minv);
  }
}

// Forward NTT column pass (global stages 0 .. logN1-1) with a tile producer;
// writes the lazy ([0, 4m)) result to buf[slot]. grid (N2/Gc, tasks).
template <int PRO>
__global__ void k_fwd_col(KArgs a, TaskList tl, const u64 *__restrict__ v, u64 *buf) {
  extern __shared__ u64 sm[];
  __shared__ u64 cst[kMaxLimbs];
  const Geo &G = a.geo;
  const int logG = log2i(G.Gc), P = pitch_of(G.Gc);
  const uint32_t w = tl.t[blockIdx.y];
  const int t = task_limb(w);
  const int c0 = blockIdx.x * G.Gc;
  produce_tile<PRO>(a, sm, cst, w, v, buf, true, logG, P, c0);
  __syncthreads();
  tile_ntt_fwd(sm, G.loga, logG, P, col_tw(a.tab.twc_f, t, G.loga), a.tab.mod[t].m);
  u64 *b = buf + (size_t)task_slot(w) * a.N;
  const int tile = 1 << (G.loga + logG);
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int y = e >> logG, g = e & ((1 << logG) - 1);
    b[((size_t)y << G.logb) + c0 + g] = sm[y * P + g];
  }
}

// Forward NTT row pass (global stages logN1 .. logN-1; all stages when N1 == 1)
// for the tile of task w, leaving canonical values in shared memory.
template <int PRO>
__device__ __forceinline__ void row_transform(const KArgs &a, u64 *sm, u64 *cst, uint32_t w,
                                              const u64 *__restrict__ v, const u64 *buf,
                                              int logG, int P, int r0) {
  const Geo &G = a.geo;
  const int t = task_limb(w);
  if (G.loga == 0)
    produce_tile<PRO>(a, sm, cst, w, v, buf, false, logG, P, r0);
  else
    produce_tile<PRO_LOAD>(a, sm, cst, w, v, buf, false, logG, P, r0);
  __syncthreads();
  tile_ntt_fwd(sm, G.logb, logG, P, row_tw(a.tab.twr_f, t, G.loga, G.logb, r0),
               a.tab.mod[t].m);
}

// Plain forward row pass: canonical result back to buf[slot].
template <int PRO>
__global__ void k_fwd_row_store(KArgs a, TaskList tl, const u64 *__restrict__ v, u64 *buf) {
  extern __shared__ u64 sm[];
  __shared__ u64 cst[kMaxLimbs];
  const Geo &G = a.geo;
  const int logG = log2i(G.Gr), P = pitch_of(G.Gr);
  const uint32_t w = tl.t[blockIdx.y];
  const int r0 = blockIdx.x * G.Gr;
  row_transform<PRO>(a, sm, cst, w, v, buf, logG, P, r0);
  const u64 m = a.tab.mod[task_limb(w)].m;
  u64 *b = buf + (size_t)task_slot(w) * a.N;
  const int tile = 1 << (G.logb + logG);
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int g = e >> G.logb, x = e & ((1 << G.logb) - 1);
    b[((size_t)(r0 + g) << G.logb) + x] = canon4(sm[x * P + g], m);
  }
}

// ModUp row pass fused with the key multiply (Sec. II-A: "each digit is then
// multiplied by the corresponding evaluation key, and the results are
// accumulated across all digits"). One CTA = one row block of one target limb t,
// looping over digits j0..j1-1:
//   acc_c[t] (+)= sum_j ext_j[t] * evk[j][c][t],  c = 0, 1
// with ext_j[t] = NTT(BConv_j)[t] (Montgomery-scaled) or, on digit j's own
// limbs, the input d_t. Sums are exact in 128 bits, reduced once by REDC.
template <int PRO>
__global__ void __launch_bounds__(512) k_fwd_row_keymult(KArgs a, TaskList tl, int j0, int j1,
                                                         SlotMap smap, int first,
                                                         const u64 *__restrict__ d,
                                                         const u64 *__restrict__ v,
                                                         const u64 *__restrict__ tmp,
                                                         const u64 *__restrict__ evk,
                                                         u64 *acc) {
  extern __shared__ u64 sm[];
  __shared__ u64 cst[kMaxLimbs];
  const Geo &G = a.geo;
  const int logG = log2i(G.Gr), P = pitch_of(G.Gr);
  const int t = task_limb(tl.t[blockIdx.y]);
  const ModInfo mi = a.tab.mod[t];
  const int r0 = blockIdx.x * G.Gr;
  const int tile = 1 << (G.logb + logG);
  const size_t N = a.N;
  U128 s0[kEPT], s1[kEPT];
#pragma unroll
  for (int k = 0; k < kEPT; ++k) s0[k] = s1[k] = U128{0, 0};
  for (int j = j0; j < j1; ++j) {
    const int lo = j * a.alpha, hi = min(lo + a.alpha, a.nq);
    const bool own = t >= lo && t < hi;
    u64 y[kEPT];
    if (own) {
#pragma unroll
      for (int k = 0; k < kEPT; ++k) {
        const int e = threadIdx.x + k * blockDim.x;
        y[k] = 0;
        if (e < tile) {
          const int g = e >> G.logb, x = e & ((1 << G.logb) - 1);
          const u64 dv = __ldg(d + (size_t)t * N + ((size_t)(r0 + g) << G.logb) + x);
          y[k] = csub(shoup(dv, mi.r1, mi.r1s, mi.m), mi.m);
        }
      }
    } else {
      const int slot = j * smap.sj + t * smap.st + smap.base;
      row_transform<PRO>(a, sm, cst, pack_task(t, j, slot), v, tmp, logG, P, r0);
#pragma unroll
      for (int k = 0; k < kEPT; ++k) {
        const int e = threadIdx.x + k * blockDim.x;
        y[k] = 0;
        if (e < tile) {
          const int g = e >> G.logb, x = e & ((1 << G.logb) - 1);
          y[k] = canon4(sm[x * P + g], mi.m);
        }
      }
      __syncthreads();
    }
    const u64 *e0 = evk + ((size_t)(j * 2 + 0) * a.qp + t) * N;
    const u64 *e1 = evk + ((size_t)(j * 2 + 1) * a.qp + t) * N;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int e = threadIdx.x + k * blockDim.x;
      if (e < tile) {
        const int g = e >> G.logb, x = e & ((1 << G.logb) - 1);
        const size_t gi = ((size_t)(r0 + g) << G.logb) + x;
        mac128(s0[k], y[k], __ldg(e0 + gi));
        mac128(s1[k], y[k], __ldg(e1 + gi));
      }
    }
  }
  u64 *a0 = acc + (size_t)t * N;
  u64 *a1 = acc + ((size_t)a.qp + t) * N;
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = threadIdx.x + k * blockDim.x;
    if (e < tile) {
      const int g = e >> G.logb, x = e & ((1 << G.logb) - 1);
      const size_t gi = ((size_t)(r0 + g) << G.logb) + x;
      u64 r0v = csub(redc(s0[k], mi.m, mi.minv), mi.m);
      u64 r1v = csub(redc(s1[k], mi.m, mi.minv), mi.m);
      if (!first) {
        r0v = addmod(r0v, a0[gi], mi.m);
        r1v = addmod(r1v, a1[gi], mi.m);
      }
      a0[gi] = r0v;
      a1[gi] = r1v;
    }
  }
}

// ModDown row pass fused with the final scaling:
//   out_c[i] = (acc_c[i] - NTT(BConv_{P->Q}(c))[i]) * P^-1 mod q_i.
// Task = (i, c, slot).
template <int PRO>
__global__ void k_fwd_row_moddown(KArgs a, TaskList tl, const u64 *__restrict__ vp,
                                  const u64 *__restrict__ tmp2, const u64 *__restrict__ acc,
                                  u64 *out) {
  extern __shared__ u64 sm[];
  __shared__ u64 cst[kMaxLimbs];
  const Geo &G = a.geo;
  const int logG = log2i(G.Gr), P = pitch_of(G.Gr);
  const uint32_t w = tl.t[blockIdx.y];
  const int i = task_limb(w), c = task_dig(w);
  const int r0 = blockIdx.x * G.Gr;
  row_transform<PRO>(a, sm, cst, w, vp, tmp2, logG, P, r0);
  const u64 m = a.tab.mod[i].m;
  const ulonglong2 pv = a.tab.pinv[i];
  const size_t N = a.N;
  const u64 *ac = acc + ((size_t)c * a.qp + i) * N;
  u64 *o = out + ((size_t)c * a.nq + i) * N;
  const int tile = 1 << (G.logb + logG);
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int g = e >> G.logb, x = e & ((1 << G.logb) - 1);
    const size_t gi = ((size_t)(r0 + g) << G.logb) + x;
    const u64 z = canon4(sm[x * P + g], m);
    o[gi] = csub(shoup(__ldg(ac + gi) + m - z, pv.x, pv.y, m), m);
  }
}

// ---------------------------------------------------------------------------
// Unfused building blocks (element-wise, coalesced; grid (N/blockDim/4, tasks)).

__global__ void k_bconv_up(KArgs a, TaskList tl, const u64 *__restrict__ v, u64 *tmp) {
  __shared__ u64 cst[kMaxLimbs];
  const uint32_t w = tl.t[blockIdx.y];
  const int t = task_limb(w), j = task_dig(w);
  const int i0 = j * a.alpha, ns = min(a.nq, i0 + a.alpha) - i0;
  stage_consts(cst, a.tab.cup + ((size_t)j * a.qp + t) * a.alpha, ns);
  __syncthreads();
  const ModInfo mi = a.tab.mod[t];
  const size_t N = a.N;
  u64 *o = tmp + (size_t)task_slot(w) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    u64 z = 0;
    int k = 0;
    while (k < ns) {
      const int kend = min(ns, k + a.run_up);
      U128 acc = {0, 0};
      for (; k < kend; ++k) mac128(acc, __ldg(v + (size_t)(i0 + k) * N + n), cst[k]);
      z = csub(z + csub(redc(acc, mi.m, mi.minv), mi.m), mi.m);
    }
    o[n] = z;
  }
}

__global__ void k_bconv_down(KArgs a, TaskList tl, const u64 *__restrict__ vp, u64 *tmp2) {
  __shared__ u64 cst[kMaxLimbs];
  const uint32_t w = tl.t[blockIdx.y];
  const int i = task_limb(w), c = task_dig(w);
  stage_consts(cst, a.tab.cdown + (size_t)i * a.alpha, a.np);
  __syncthreads();
  const ModInfo mi = a.tab.mod[i];
  const size_t N = a.N;
  const u64 *src = vp + (size_t)c * a.np * N;
  u64 *o = tmp2 + (size_t)task_slot(w) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    u64 z = 0;
    int k = 0;
    while (k < a.np) {
      const int kend = min(a.np, k + a.run_down);
      U128 acc = {0, 0};
      for (; k < kend; ++k) mac128(acc, __ldg(src + (size_t)k * N + n), cst[k]);
      z = csub(z + csub(redc(acc, mi.m, mi.minv), mi.m), mi.m);
    }
    o[n] = z;
  }
}

__global__ void k_keymult(KArgs a, TaskList tl, int j0, int j1, SlotMap smap, int first,
                          const u64 *__restrict__ d, const u64 *__restrict__ tmp,
                          const u64 *__restrict__ evk, u64 *acc) {
  const int t = task_limb(tl.t[blockIdx.y]);
  const ModInfo mi = a.tab.mod[t];
  const size_t N = a.N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    U128 s0 = {0, 0}, s1 = {0, 0};
    for (int j = j0; j < j1; ++j) {
      const int lo = j * a.alpha, hi = min(lo + a.alpha, a.nq);
      u64 y;
      if (t >= lo && t < hi)
        y = csub(shoup(__ldg(d + (size_t)t * N + n), mi.r1, mi.r1s, mi.m), mi.m);
      else
        y = __ldg(tmp + (size_t)(j * smap.sj + t * smap.st + smap.base) * N + n);
      mac128(s0, y, __ldg(evk + ((size_t)(j * 2 + 0) * a.qp + t) * N + n));
      mac128(s1, y, __ldg(evk + ((size_t)(j * 2 + 1) * a.qp + t) * N + n));
    }
    u64 r0v = csub(redc(s0, mi.m, mi.minv), mi.m);
    u64 r1v = csub(redc(s1, mi.m, mi.minv), mi.m);
    u64 *a0 = acc + (size_t)t * N + n;
    u64 *a1 = acc + ((size_t)a.qp + t) * N + n;
    if (!first) {
      r0v = addmod(r0v, *a0, mi.m);
      r1v = addmod(r1v, *a1, mi.m);
    }
    *a0 = r0v;
    *a1 = r1v;
  }
}

__global__ void k_moddown_scale(KArgs a, TaskList tl, const u64 *__restrict__ tmp2,
                                const u64 *__restrict__ acc, u64 *out) {
  const uint32_t w = tl.t[blockIdx.y];
  const int i = task_limb(w), c = task_dig(w);
  const u64 m = a.tab.mod[i].m;
  const ulonglong2 pv = a.tab.pinv[i];
  const size_t N = a.N;
  const u64 *z = tmp2 + (size_t)task_slot(w) * N;
  const u64 *ac = acc + ((size_t)c * a.qp + i) * N;
  u64 *o = out + ((size_t)c * a.nq + i) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x)
    o[n] = csub(shoup(__ldg(ac + n) + m - __ldg(z + n), pv.x, pv.y, m), m);
}

// ---------------------------------------------------------------------------
// Key generation helpers.
// polys layout [2 + beta][QP][N]: 0 = s_from, 1 = s_to, 2 + j = e_j, as residues.
__global__ void k_keygen_lift(KArgs a, const int8_t *__restrict__ sf,
                              const int8_t *__restrict__ st, const int32_t *__restrict__ e,
                              u64 *polys) {
  const int poly = blockIdx.z, t = blockIdx.y;
  const u64 m = a.tab.mod[t].m;
  const size_t N = a.N;
  u64 *o = polys + ((size_t)poly * a.qp + t) * N;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N;
       n += (size_t)gridDim.x * blockDim.x) {
    long long x;
    if (poly == 0)
      x = sf[n];
    else if (poly == 1)
      x = st[n];
    else
      x = e[(size_t)(poly - 2) * N + n];
    u64 r = (u64)(x < 0 ? -x : x) % m;
    o[n] = (x < 0 && r) ? m - r : r;
  }
}

__device__ __forceinline__ u64 mulmod_full(u64 x, u64 y, const ModInfo &mi, u64 r2) {
  U128 p = {0, 0};
  mac128(p, x, y);
  const u64 t = csub(redc(p, mi.m, mi.minv), mi.m);  // x y 2^-64
  U128 p2 = {0, 0};
  mac128(p2, t, r2);
  return csub(redc(p2, mi.m, mi.minv), mi.m);  // x y
}

// evk[j][0][t] = -a_j s_to + e_j + [P g_j]_t s_from; evk[j][1][t] = a_j.
__global__ void k_keygen_combine(KArgs a, const u64 *__restrict__ polys,
                                 const u64 *__restrict__ arand, u64 *evk) {
  const int j = blockIdx.z, t = blockIdx.y;
  const ModInfo mi = a.tab.mod[t];
  const u64 m = mi.m, r2 = mi.r2;
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
    const u64 as = mulmod_full(av, st[n], mi, r2);
    v = v >= as ? v - as : v + m - as;
    v = addmod(v, mulmod_full(pg, sf[n], mi, r2), m);
    b[n] = v;
    ao[n] = av;
  }
}

size_t col_smem(const Geo &g) { return ((size_t)1 << g.loga) * (g.Gc + 1) * 8; }
size_t row_smem(const Geo &g) {
  return ((size_t)1 << g.logb) * (g.Gr == 1 ? 1 : g.Gr + 1) * 8;
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
  return cudaSuccess;
}

int ew_blocks(size_t N) {
  size_t b = (N + 1023) / 1024;
  return (int)(b < 1 ? 1 : b);
}

// Split a task list into launches of at most kMaxTasks entries (gridDim.y).
template <class F>
cudaError_t for_each_part(const TaskList &tl, F f) {
  if (tl.n <= 0) return cudaSuccess;
  for (int s = 0; s < tl.n; s += kMaxTasks) {
    TaskList part;
    part.n = tl.n - s < kMaxTasks ? tl.n - s : kMaxTasks;
    for (int k = 0; k < part.n; ++k) part.t[k] = tl.t[s + k];
    f(part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers

cudaError_t launch_intt(const ks_context *c, const u64 *src, int src_outer, u64 *dst,
                        int dst_outer, int outer, int inner, int prime_base,
                        const ulonglong2 *scale, u64 * /*mid*/, cudaStream_t s) {
  if (outer * inner == 0) return cudaSuccess;
  const KArgs a = make_args(c);
  const Geo &g = c->geo;
  const size_t rs = row_smem(g);
  cudaError_t e = set_smem(k_inv_row, rs);
  if (e) return e;
  dim3 gr((1 << g.loga) / g.Gr, outer * inner);
  k_inv_row<<<gr, g.ntr, rs, s>>>(a, src, src_outer, dst, dst_outer, inner, prime_base, scale);
  if ((e = cudaGetLastError())) return e;
  if (g.loga == 0) return cudaSuccess;
  const size_t cs = col_smem(g);
  if ((e = set_smem(k_inv_col, cs))) return e;
  dim3 gc((1 << g.logb) / g.Gc, outer * inner);
  k_inv_col<<<gc, g.ntc, cs, s>>>(a, dst, dst_outer, inner, prime_base, scale);
  return cudaGetLastError();
}

cudaError_t launch_modup_col(const ks_context *c, const TaskList &tl, const u64 *v, u64 *tmp,
                             cudaStream_t s) {
  const Geo &g = c->geo;
  if (g.loga == 0) return cudaSuccess;
  const KArgs a = make_args(c);
  const size_t cs = col_smem(g);
  cudaError_t e = set_smem(k_fwd_col<PRO_UP>, cs);
  if (e) return e;
  return for_each_part(tl, [&](const TaskList &p) {
    dim3 gc((1 << g.logb) / g.Gc, p.n);
    k_fwd_col<PRO_UP><<<gc, g.ntc, cs, s>>>(a, p, v, tmp);
  });
}

cudaError_t launch_modup_row(const ks_context *c, const int *targets, int ntargets, int j0,
                             int j1, SlotMap smap, bool first, const u64 *d, const u64 *v,
                             const u64 *tmp, const u64 *evk, u64 *acc, cudaStream_t s) {
  if (ntargets == 0) return cudaSuccess;
  const KArgs a = make_args(c);
  const Geo &g = c->geo;
  const size_t rs = row_smem(g);
  TaskList tl;
  tl.n = ntargets;
  for (int k = 0; k < ntargets; ++k) tl.t[k] = pack_task(targets[k], 0, 0);
  dim3 gr((1 << g.loga) / g.Gr, ntargets);
  cudaError_t e;
  if (g.loga == 0) {
    if ((e = set_smem(k_fwd_row_keymult<PRO_UP>, rs))) return e;
    k_fwd_row_keymult<PRO_UP><<<gr, g.ntr, rs, s>>>(a, tl, j0, j1, smap, first ? 1 : 0, d, v,
                                                    tmp, evk, acc);
  } else {
    if ((e = set_smem(k_fwd_row_keymult<PRO_LOAD>, rs))) return e;
    k_fwd_row_keymult<PRO_LOAD><<<gr, g.ntr, rs, s>>>(a, tl, j0, j1, smap, first ? 1 : 0, d, v,
                                                      tmp, evk, acc);
  }
  return cudaGetLastError();
}

cudaError_t launch_moddown_col(const ks_context *c, const TaskList &tl, const u64 *vp,
                               u64 *tmp2, cudaStream_t s) {
  const Geo &g = c->geo;
  if (g.loga == 0) return cudaSuccess;
  const KArgs a = make_args(c);
  const size_t cs = col_smem(g);
  cudaError_t e = set_smem(k_fwd_col<PRO_DOWN>, cs);
  if (e) return e;
  return for_each_part(tl, [&](const TaskList &p) {
    dim3 gc((1 << g.logb) / g.Gc, p.n);
    k_fwd_col<PRO_DOWN><<<gc, g.ntc, cs, s>>>(a, p, vp, tmp2);
  });
}

cudaError_t launch_moddown_row(const ks_context *c, const TaskList &tl, const u64 *vp,
                               const u64 *tmp2, const u64 *acc, u64 *out, cudaStream_t s) {
  const KArgs a = make_args(c);
  const Geo &g = c->geo;
  const size_t rs = row_smem(g);
  cudaError_t e;
  if (g.loga == 0) {
    if ((e = set_smem(k_fwd_row_moddown<PRO_DOWN>, rs))) return e;
  } else {
    if ((e = set_smem(k_fwd_row_moddown<PRO_LOAD>, rs))) return e;
  }
  return for_each_part(tl, [&](const TaskList &p) {
    dim3 gr((1 << g.loga) / g.Gr, p.n);
    if (g.loga == 0)
      k_fwd_row_moddown<PRO_DOWN><<<gr, g.ntr, rs, s>>>(a, p, vp, tmp2, acc, out);
    else
      k_fwd_row_moddown<PRO_LOAD><<<gr, g.ntr, rs, s>>>(a, p, vp, tmp2, acc, out);
  });
}

cudaError_t launch_bconv_up(const ks_context *c, const TaskList &tl, const u64 *v, u64 *tmp,
                            cudaStream_t s) {
  const KArgs a = make_args(c);
  return for_each_part(tl, [&](const TaskList &p) {
    k_bconv_up<<<dim3(ew_blocks(c->N), p.n), 256, 0, s>>>(a, p, v, tmp);
  });
}

cudaError_t launch_bconv_down(const ks_context *c, const TaskList &tl, const u64 *vp,
                              u64 *tmp2, cudaStream_t s) {
  const KArgs a = make_args(c);
  return for_each_part(tl, [&](const TaskList &p) {
    k_bconv_down<<<dim3(ew_blocks(c->N), p.n), 256, 0, s>>>(a, p, vp, tmp2);
  });
}

cudaError_t launch_ntt_plain(const ks_context *c, const TaskList &tl, u64 *buf, u64 * /*mid*/,
                             cudaStream_t s) {
  const KArgs a = make_args(c);
  const Geo &g = c->geo;
  cudaError_t e;
  if (g.loga > 0) {
    const size_t cs = col_smem(g);
    if ((e = set_smem(k_fwd_col<PRO_LOAD>, cs))) return e;
    e = for_each_part(tl, [&](const TaskList &p) {
      k_fwd_col<PRO_LOAD><<<dim3((1 << g.logb) / g.Gc, p.n), g.ntc, cs, s>>>(a, p, nullptr,
                                                                             buf);
    });
    if (e) return e;
  }
  const size_t rs = row_smem(g);
  if ((e = set_smem(k_fwd_row_store<PRO_LOAD>, rs))) return e;
  return for_each_part(tl, [&](const TaskList &p) {
    k_fwd_row_store<PRO_LOAD><<<dim3((1 << g.loga) / g.Gr, p.n), g.ntr, rs, s>>>(a, p, nullptr,
                                                                                 buf);
  });
}

cudaError_t launch_keymult(const ks_context *c, const int *targets, int ntargets, int j0,
                           int j1, SlotMap smap, bool first, const u64 *d, const u64 *tmp,
                           const u64 *evk, u64 *acc, cudaStream_t s) {
  if (ntargets == 0) return cudaSuccess;
  const KArgs a = make_args(c);
  TaskList tl;
  tl.n = ntargets;
  for (int k = 0; k < ntargets; ++k) tl.t[k] = pack_task(targets[k], 0, 0);
  k_keymult<<<dim3(ew_blocks(c->N), ntargets), 256, 0, s>>>(a, tl, j0, j1, smap, first ? 1 : 0,
                                                            d, tmp, evk, acc);
  return cudaGetLastError();
}

cudaError_t launch_moddown_scale(const ks_context *c, const TaskList &tl, const u64 *tmp2,
                                 const u64 *acc, u64 *out, cudaStream_t s) {
  const KArgs a = make_args(c);
  return for_each_part(tl, [&](const TaskList &p) {
    k_moddown_scale<<<dim3(ew_blocks(c->N), p.n), 256, 0, s>>>(a, p, tmp2, acc, out);
  });
}

cudaError_t launch_keygen_lift(const ks_context *c, const int8_t *sf, const int8_t *st,
                               const int32_t *e, u64 *polys, cudaStream_t s) {
  const KArgs a = make_args(c);
  k_keygen_lift<<<dim3(ew_blocks(c->N), c->qp, 2 + c->beta), 256, 0, s>>>(a, sf, st, e, polys);
  return cudaGetLastError();
}

cudaError_t launch_keygen_combine(const ks_context *c, const u64 *polys, const u64 *arand,
                                  u64 *evk, cudaStream_t s) {
  const KArgs a = make_args(c);
  k_keygen_combine<<<dim3(ew_blocks(c->N), c->qp, c->beta), 256, 0, s>>>(a, polys, arand, evk);
  return cudaGetLastError();
}

}  // namespace ks
