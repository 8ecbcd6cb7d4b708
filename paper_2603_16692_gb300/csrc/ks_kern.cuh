// KeySwitch kernel templates for sm_103a, specialised per N = 2^LOGN (included by
// the ks_inst_*.cu instantiation units).
//
// Two-pass negacyclic NTT / iNTT (column pass, row pass) with the fast basis
// conversions fused into the first forward pass and the key multiply or the
// ModDown scaling fused into the last one (Sec. II-A, Fig. 1). Twiddles of a tile
// are staged into shared memory once per CTA and reused for every polynomial the
// CTA transforms (all digits of a target limb; both accumulators in ModDown).
#pragma once
#include <cuda_runtime.h>

#include "ks_arith.cuh"
#include "ks_internal.h"
#include "ks_ntt.cuh"

namespace ks {
namespace kern {

enum { PRO_LOAD = 0, PRO_UP = 1, PRO_DOWN = 2 };

struct KArgs {
  Tables tab;
  int N, nq, np, qp, alpha, beta;
  int run_up, run_down;
};

inline KArgs make_args(const ks_context *c) {
  KArgs a;
  a.tab = c->tab;
  a.N = c->N;
  a.nq = c->nq;
  a.np = c->np;
  a.qp = c->qp;
  a.alpha = c->alpha;
  a.beta = c->beta;
  a.run_up = c->run_up;
  a.run_down = c->run_down;
  return a;
}

// ---------------------------------------------------------------------------
// Tile movement. Rows r0..r0+G-1 of a limb are contiguous; columns c0..c0+G-1
// are G contiguous words in each of the N1 rows. 16-byte vector accesses,
// plain (coherent) loads: some kernels transform a buffer in place.

template <class GT>
__device__ __forceinline__ void load_rows(u64 *s, const u64 *src, int r0) {
  constexpr int TILE = GT::TILE, LOGB = GT::LOGB, P = GT::PR;
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src + ((size_t)r0 << LOGB));
#pragma unroll
  for (int it = 0; it < (TILE / 2 + GT::NT - 1) / GT::NT; ++it) {
    const int e2 = threadIdx.x + it * GT::NT;
    if ((TILE / 2) % GT::NT != 0 && e2 >= TILE / 2) break;
    const ulonglong2 val = s2[e2];
    const int e = 2 * e2, g = e >> LOGB, x = e & ((1 << LOGB) - 1);
    s[x * P + g] = val.x;
    s[(x + 1) * P + g] = val.y;
  }
}

template <class GT>
__device__ __forceinline__ void store_rows(u64 *dst, const u64 *s, int r0, u64 m, int mode) {
  // mode 0: as is; 1: [0,4m) -> canonical
  constexpr int TILE = GT::TILE, LOGB = GT::LOGB, P = GT::PR;
  ulonglong2 *d2 = reinterpret_cast<ulonglong2 *>(dst + ((size_t)r0 << LOGB));
#pragma unroll
  for (int it = 0; it < (TILE / 2 + GT::NT - 1) / GT::NT; ++it) {
    const int e2 = threadIdx.x + it * GT::NT;
    if ((TILE / 2) % GT::NT != 0 && e2 >= TILE / 2) break;
    const int e = 2 * e2, g = e >> LOGB, x = e & ((1 << LOGB) - 1);
    ulonglong2 val;
    val.x = s[x * P + g];
    val.y = s[(x + 1) * P + g];
    if (mode == 1) {
      val.x = canon4(val.x, m);
      val.y = canon4(val.y, m);
    }
    d2[e2] = val;
  }
}

template <class GT>
__device__ __forceinline__ void load_cols(u64 *s, const u64 *src, int c0) {
  constexpr int TILE = GT::N1 * GT::GC, LOGG = GT::LOGGC, P = GT::PC;
#pragma unroll
  for (int it = 0; it < (TILE / 2 + GT::NT - 1) / GT::NT; ++it) {
    const int e2 = threadIdx.x + it * GT::NT;
    if ((TILE / 2) % GT::NT != 0 && e2 >= TILE / 2) break;
    const int e = 2 * e2, y = e >> LOGG, g = e & ((1 << LOGG) - 1);
    const ulonglong2 val =
        *reinterpret_cast<const ulonglong2 *>(src + ((size_t)y << GT::LOGB) + c0 + g);
    s[y * P + g] = val.x;
    s[y * P + g + 1] = val.y;
  }
}

template <class GT>
__device__ __forceinline__ void store_cols(u64 *dst, const u64 *s, int c0) {
  constexpr int TILE = GT::N1 * GT::GC, LOGG = GT::LOGGC, P = GT::PC;
#pragma unroll
  for (int it = 0; it < (TILE / 2 + GT::NT - 1) / GT::NT; ++it) {
    const int e2 = threadIdx.x + it * GT::NT;
    if ((TILE / 2) % GT::NT != 0 && e2 >= TILE / 2) break;
    const int e = 2 * e2, y = e >> LOGG, g = e & ((1 << LOGG) - 1);
    ulonglong2 val;
    val.x = s[y * P + g];
    val.y = s[y * P + g + 1];
    *reinterpret_cast<ulonglong2 *>(dst + ((size_t)y << GT::LOGB) + c0 + g) = val;
  }
}

// Stage n twiddle pairs into shared memory.
template <class GT>
__device__ __forceinline__ void stage_tw(ulonglong2 *tws, const ulonglong2 *__restrict__ src,
                                         int n) {
  for (int k = threadIdx.x; k < n; k += GT::NT) tws[k] = __ldg(src + k);
}

// Column-pass twiddles of a prime: the first N1 entries of its column table.
template <class GT>
__device__ __forceinline__ const ulonglong2 *col_table(const ulonglong2 *tab, int prime) {
  return tab + ((size_t)prime << GT::LOGA);
}
// Row-pass twiddle slab of (prime, row tile blk): (N2-1)*GR entries, stage-major.
template <class GT>
__device__ __forceinline__ const ulonglong2 *row_table(const ulonglong2 *tab, int prime,
                                                       int blk) {
  return tab + (size_t)prime * (GT::N2 - 1) * GT::N1 + (size_t)blk * GT::TWR;
}

__device__ __forceinline__ void stage_consts(u64 *cst, const u64 *__restrict__ src, int n,
                                             int nt) {
  for (int k = threadIdx.x; k < n; k += nt) cst[k] = __ldg(src + k);
}

// Fast basis conversion into a tile: element -> REDC(sum_k src_k[gidx] * cst[k]),
// in runs of at most `run` terms per exact 128-bit sum. Output in [0, 2m).
// COL: column tile (element (y, g) = limb index y*N2 + base + g);
// otherwise row tile (element (x, g) = limb index (base + g)*N2 + x).
template <class GT, bool COL>
__device__ __forceinline__ void bconv_tile(u64 *s, const u64 *__restrict__ src, size_t N,
                                           int nsrc, const u64 *cst, int run, int base, u64 m,
                                           u64 minv) {
  constexpr int LOGG = COL ? GT::LOGGC : GT::LOGGR;
  constexpr int TILE = COL ? GT::N1 * GT::GC : GT::N2 * GT::GR;
  constexpr int P = COL ? GT::PC : GT::PR;
  constexpr int EPT = (TILE + GT::NT - 1) / GT::NT;
  constexpr int H = EPT >= 4 ? 4 : EPT;  // elements per batch (bounds live registers)
  const u64 m2 = 2 * m;
#pragma unroll 1
  for (int k0 = 0; k0 < EPT; k0 += H) {
    int gi[H];
    U128 acc[H];
    u64 z[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int e = threadIdx.x + (k0 + k) * GT::NT;
      if (COL) {
        const int y = e >> LOGG, g = e & ((1 << LOGG) - 1);
        gi[k] = (y << GT::LOGB) + base + g;
      } else {
        const int g = e >> GT::LOGB, x = e & ((1 << GT::LOGB) - 1);
        gi[k] = ((base + g) << GT::LOGB) + x;
      }
      acc[k] = U128{0, 0};
      z[k] = 0;
    }
    int cnt = 0;
    for (int i = 0; i < nsrc; ++i) {
      const u64 c = cst[i];
      const u64 *si = src + (size_t)i * N;
      u64 x[H];
#pragma unroll
      for (int k = 0; k < H; ++k)
        x[k] = (TILE % GT::NT == 0 || threadIdx.x + (k0 + k) * GT::NT < TILE) ? __ldg(si + gi[k])
                                                                             : 0;
#pragma unroll
      for (int k = 0; k < H; ++k) mac128(acc[k], x[k], c);
      if (++cnt == run || i == nsrc - 1) {
#pragma unroll
        for (int k = 0; k < H; ++k) {
          const u64 zz = z[k] + redc(acc[k], m, minv);
          z[k] = zz >= m2 ? zz - m2 : zz;
          acc[k] = U128{0, 0};
        }
        cnt = 0;
      }
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int e = threadIdx.x + (k0 + k) * GT::NT;
      if (TILE % GT::NT != 0 && e >= TILE) break;
      const int sidx = COL ? (e >> LOGG) * P + (e & ((1 << LOGG) - 1))
                           : (e & ((1 << GT::LOGB) - 1)) * P + (e >> GT::LOGB);
      s[sidx] = z[k];
    }
  }
}

// Produce the tile of task w: BConv (ModUp: digit j onto limb t, Montgomery-scaled
// by constants carrying 2^128; ModDown: P-limbs of polynomial c onto q_i) or a
// plain load of buf[slot].
template <class GT, int PRO, bool COL>
__device__ __forceinline__ void produce(const KArgs &a, u64 *sm, u64 *cst, uint32_t w,
                                        const u64 *__restrict__ v, const u64 *buf, int base) {
  const int t = task_limb(w);
  const size_t N = a.N;
  if (PRO == PRO_LOAD) {
    const u64 *b = buf + (size_t)task_slot(w) * N;
    if (COL)
      load_cols<GT>(sm, b, base);
    else
      load_rows<GT>(sm, b, base);
  } else if (PRO == PRO_UP) {
    const int j = task_dig(w);
    const int i0 = j * a.alpha;
    const int ns = min(a.nq, i0 + a.alpha) - i0;
    stage_consts(cst, a.tab.cup + ((size_t)j * a.qp + t) * a.alpha, ns, GT::NT);
    __syncthreads();
    const ModInfo mi = a.tab.mod[t];
    bconv_tile<GT, COL>(sm, v + (size_t)i0 * N, N, ns, cst, a.run_up, base, mi.m, mi.minv);
  } else {
    const int c = task_dig(w);
    stage_consts(cst, a.tab.cdown + (size_t)t * a.alpha, a.np, GT::NT);
    __syncthreads();
    const ModInfo mi = a.tab.mod[t];
    bconv_tile<GT, COL>(sm, v + (size_t)c * a.np * N, N, a.np, cst, a.run_down, base, mi.m,
                        mi.minv);
  }
}

// Shared-memory layout of the kernels: twiddles first (16-byte aligned), then
// the tile.
template <class GT, bool COL>
__device__ __forceinline__ u64 *tile_ptr(unsigned char *raw) {
  return reinterpret_cast<u64 *>(raw + (COL ? GT::TWC : GT::TWR) * 16);
}

// ---------------------------------------------------------------------------
// Inverse NTT, row pass (global stages logN-1 .. logN1), for `outer` polynomials
// of the same limb (src + (o*src_outer + ii)*N). grid (N1/GR, inner). With a
// single pass (N1 == 1) it also applies the per-limb scale (canonical output).
template <int LOGN>
__global__ void __launch_bounds__(GeoT<LOGN>::NT)
    k_inv_row(KArgs a, const u64 *src, int src_outer, u64 *dst, int dst_outer, int outer,
              int prime_base, const ulonglong2 *__restrict__ scale) {
  using GT = GeoT<LOGN>;
  extern __shared__ __align__(16) unsigned char raw[];
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const int ii = blockIdx.y, prime = prime_base + ii, blk = blockIdx.x;
  const int r0 = blk * GT::GR;
  const u64 m = a.tab.mod[prime].m;
  const size_t N = a.N;
  stage_tw<GT>(tws, row_table<GT>(a.tab.twr_i, prime, blk), GT::TWR);
  const ulonglong2 sc = scale[ii];
  for (int o = 0; o < outer; ++o) {
    load_rows<GT>(sm, src + ((size_t)o * src_outer + ii) * N, r0);
    __syncthreads();
    tile_inv<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true>(sm, tws, m);
    u64 *d = dst + ((size_t)o * dst_outer + ii) * N;
    if (GT::LOGA == 0) {
#pragma unroll
      for (int k = 0; k < GT::EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT != 0 && e >= GT::TILE) break;
        d[e] = csub(shoup(sm[e], sc.x, sc.y, m), m);
      }
    } else {
      store_rows<GT>(d, sm, r0, m, 0);
    }
    __syncthreads();
  }
}

// Inverse NTT, column pass (global stages logN1-1 .. 0), in place, then the
// per-limb scale. grid (N2/GC, inner).
template <int LOGN>
__global__ void __launch_bounds__(GeoT<LOGN>::NT, 2048 / GeoT<LOGN>::NT / 2)
    k_inv_col(KArgs a, u64 *dst, int dst_outer, int outer, int prime_base,
              const ulonglong2 *__restrict__ scale) {
  using GT = GeoT<LOGN>;
  extern __shared__ __align__(16) unsigned char raw[];
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, true>(raw);
  const int ii = blockIdx.y, prime = prime_base + ii;
  const int c0 = blockIdx.x * GT::GC;
  const u64 m = a.tab.mod[prime].m;
  stage_tw<GT>(tws, col_table<GT>(a.tab.twc_i, prime), GT::TWC);
  const ulonglong2 sc = scale[ii];
  for (int o = 0; o < outer; ++o) {
    u64 *d = dst + ((size_t)o * dst_outer + ii) * (size_t)a.N;
    load_cols<GT>(sm, d, c0);
    __syncthreads();
    tile_inv<GT::LOGA, GT::LOGGC, GT::PC, GT::NT, false>(sm, tws, m);
    constexpr int TILE = GT::N1 * GT::GC;
#pragma unroll
    for (int k = 0; k < (TILE + GT::NT - 1) / GT::NT; ++k) {
      const int e = threadIdx.x + k * GT::NT;
      if (TILE % GT::NT != 0 && e >= TILE) break;
      const int y = e >> GT::LOGGC, g = e & (GT::GC - 1);
      sm[y * GT::PC + g] = csub(shoup(sm[y * GT::PC + g], sc.x, sc.y, m), m);
    }
    __syncthreads();
    store_cols<GT>(d, sm, c0);
    __syncthreads();
  }
}

// Forward NTT, column pass (global stages 0 .. logN1-1) with a tile producer;
// the lazy ([0, 4m)) result goes to buf[slot]. grid (N2/GC, tasks).
template <int LOGN, int PRO>
__global__ void __launch_bounds__(GeoT<LOGN>::NT)
    k_fwd_col(KArgs a, TaskList tl, const u64 *__restrict__ v, u64 *buf) {
  using GT = GeoT<LOGN>;
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ u64 cst[kMaxLimbs];
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, true>(raw);
  const uint32_t w = tl.t[blockIdx.y];
  const int t = task_limb(w);
  const int c0 = blockIdx.x * GT::GC;
  stage_tw<GT>(tws, col_table<GT>(a.tab.twc_f, t), GT::TWC);
  produce<GT, PRO, true>(a, sm, cst, w, v, buf, c0);
  __syncthreads();
  tile_fwd<GT::LOGA, GT::LOGGC, GT::PC, GT::NT, false>(sm, tws, a.tab.mod[t].m);
  store_cols<GT>(buf + (size_t)task_slot(w) * a.N, sm, c0);
}

// Plain forward row pass: canonical result back to buf[slot]. grid (N1/GR, tasks).
template <int LOGN>
__global__ void __launch_bounds__(GeoT<LOGN>::NT) k_fwd_row_store(KArgs a, TaskList tl, u64 *buf) {
  using GT = GeoT<LOGN>;
  extern __shared__ __align__(16) unsigned char raw[];
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const uint32_t w = tl.t[blockIdx.y];
  const int t = task_limb(w), blk = blockIdx.x, r0 = blk * GT::GR;
  const u64 m = a.tab.mod[t].m;
  stage_tw<GT>(tws, row_table<GT>(a.tab.twr_f, t, blk), GT::TWR);
  u64 *b = buf + (size_t)task_slot(w) * a.N;
  load_rows<GT>(sm, b, r0);
  __syncthreads();
  tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true>(sm, tws, m);
  store_rows<GT>(b, sm, r0, m, 1);
}

// ModUp row pass fused with the key multiply. One CTA = one row tile of one
// target limb t, over digits j0..j1-1:
//   acc_c[t] (+)= sum_j ext_j[t] * evk[j][c][t],  c = 0, 1,
// with ext_j[t] = NTT(BConv_j)[t] (Montgomery-scaled) or, on digit j's own limbs,
// the input d_t (put in Montgomery form here), so that REDC of each exact
// 128-bit product is the plain product mod m. The row twiddles of (t, tile) are
// staged once.
template <int LOGN, int PRO>
__global__ void __launch_bounds__(GeoT<LOGN>::NT, 2048 / GeoT<LOGN>::NT / 8 * 3)
    k_fwd_row_keymult(KArgs a, TaskList tl, int j0, int j1, SlotMap smap, int first,
                      const u64 *__restrict__ d, const u64 *__restrict__ v,
                      const u64 *__restrict__ tmp, const u64 *__restrict__ evk, u64 *acc) {
  using GT = GeoT<LOGN>;
  constexpr int EPT = GT::EPT;
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ u64 cst[kMaxLimbs];
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const int t = task_limb(tl.t[blockIdx.y]);
  const ModInfo mi = a.tab.mod[t];
  const int blk = blockIdx.x, r0 = blk * GT::GR;
  const size_t N = a.N;
  const size_t off0 = (size_t)r0 << GT::LOGB;  // the tile is contiguous from here
  stage_tw<GT>(tws, row_table<GT>(a.tab.twr_f, t, blk), GT::TWR);
  // Per-digit products are reduced by REDC and summed lazily in [0, 2m).
  u64 s0[EPT], s1[EPT];
  const u64 m2 = 2 * mi.m;
#pragma unroll
  for (int k = 0; k < EPT; ++k) s0[k] = s1[k] = 0;
  for (int j = j0; j < j1; ++j) {
    const int lo = j * a.alpha, hi = min(lo + a.alpha, a.nq);
    const bool own = t >= lo && t < hi;
    const u64 *e0 = evk + ((size_t)(j * 2 + 0) * a.qp + t) * N + off0;
    const u64 *e1 = evk + ((size_t)(j * 2 + 1) * a.qp + t) * N + off0;
    if (own) {
      const u64 *dt = d + (size_t)t * N + off0;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT == 0 || e < GT::TILE) {
          const u64 y = csub(shoup(__ldg(dt + e), mi.r1, mi.r1s, mi.m), mi.m);
          U128 p0 = {0, 0}, p1 = {0, 0};
          mac128(p0, y, __ldg(e0 + e));
          mac128(p1, y, __ldg(e1 + e));
          const u64 a0v = s0[k] + redc(p0, mi.m, mi.minv), a1v = s1[k] + redc(p1, mi.m, mi.minv);
          s0[k] = a0v >= m2 ? a0v - m2 : a0v;
          s1[k] = a1v >= m2 ? a1v - m2 : a1v;
        }
      }
    } else {
      const int slot = j * smap.sj + t * smap.st + smap.base;
      if (GT::LOGA == 0)
        produce<GT, PRO, false>(a, sm, cst, pack_task(t, j, slot), v, tmp, r0);
      else
        produce<GT, PRO_LOAD, false>(a, sm, cst, pack_task(t, j, slot), v, tmp, r0);
      __syncthreads();
      tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true>(sm, tws, mi.m);
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT == 0 || e < GT::TILE) {
          const int g = e >> GT::LOGB, x = e & (GT::N2 - 1);
          const u64 y = canon4(sm[x * GT::PR + g], mi.m);
          U128 p0 = {0, 0}, p1 = {0, 0};
          mac128(p0, y, __ldg(e0 + e));
          mac128(p1, y, __ldg(e1 + e));
          const u64 a0v = s0[k] + redc(p0, mi.m, mi.minv), a1v = s1[k] + redc(p1, mi.m, mi.minv);
          s0[k] = a0v >= m2 ? a0v - m2 : a0v;
          s1[k] = a1v >= m2 ? a1v - m2 : a1v;
        }
      }
      __syncthreads();
    }
  }
  u64 *a0 = acc + (size_t)t * N + off0;
  u64 *a1 = acc + ((size_t)a.qp + t) * N + off0;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = threadIdx.x + k * GT::NT;
    if (GT::TILE % GT::NT != 0 && e >= GT::TILE) break;
    u64 r0v = csub(s0[k], mi.m);
    u64 r1v = csub(s1[k], mi.m);
    if (!first) {
      r0v = addmod(r0v, a0[e], mi.m);
      r1v = addmod(r1v, a1[e], mi.m);
    }
    a0[e] = r0v;
    a1[e] = r1v;
  }
}

// ModDown row pass fused with the final scaling, both polynomials c = 0, 1 of
// limb i in one CTA (shared twiddles):
//   out_c[i] = (acc_c[i] - NTT(BConv_{P->Q}(c))[i]) * P^-1 mod q_i.
// Task = (i, slot of c = 0); polynomial c uses slot + c*span.
template <int LOGN, int PRO>
__global__ void __launch_bounds__(GeoT<LOGN>::NT)
    k_fwd_row_moddown(KArgs a, TaskList tl, int span, const u64 *__restrict__ vp,
                      const u64 *__restrict__ tmp2, const u64 *__restrict__ acc, u64 *out) {
  using GT = GeoT<LOGN>;
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ u64 cst[kMaxLimbs];
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const uint32_t w = tl.t[blockIdx.y];
  const int i = task_limb(w), blk = blockIdx.x, r0 = blk * GT::GR;
  const u64 m = a.tab.mod[i].m;
  const ulonglong2 pv = a.tab.pinv[i];
  const size_t N = a.N;
  const size_t off0 = (size_t)r0 << GT::LOGB;
  stage_tw<GT>(tws, row_table<GT>(a.tab.twr_f, i, blk), GT::TWR);
  for (int c = 0; c < 2; ++c) {
    const uint32_t wc = pack_task(i, c, task_slot(w) + c * span);
    if (GT::LOGA == 0)
      produce<GT, PRO, false>(a, sm, cst, wc, vp, tmp2, r0);
    else
      produce<GT, PRO_LOAD, false>(a, sm, cst, wc, vp, tmp2, r0);
    __syncthreads();
    tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true>(sm, tws, m);
    const u64 *ac = acc + ((size_t)c * a.qp + i) * N + off0;
    u64 *o = out + ((size_t)c * a.nq + i) * N + off0;
#pragma unroll
    for (int k = 0; k < GT::EPT; ++k) {
      const int e = threadIdx.x + k * GT::NT;
      if (GT::TILE % GT::NT != 0 && e >= GT::TILE) break;
      const int g = e >> GT::LOGB, x = e & (GT::N2 - 1);
      const u64 z = canon4(sm[x * GT::PR + g], m);
      o[e] = csub(shoup(__ldg(ac + e) + m - z, pv.x, pv.y, m), m);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers for one N.

// Opt in to the kernel's dynamic shared memory (static shared memory such as the
// BConv constants comes on top of it) and to the largest shared-memory carveout,
// once per kernel.
cudaError_t smem_opt_in(const void *kernel, int bytes);

template <class K>
inline cudaError_t smem_attr(K kernel, int bytes) {
  return smem_opt_in(reinterpret_cast<const void *>(kernel), bytes);
}

template <class F>
inline cudaError_t for_each_part(const TaskList &tl, F f) {
  if (tl.n <= 0) return cudaSuccess;
  if (tl.n <= kMaxTasks) {
    f(tl);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

template <int LOGN>
struct Launch {
  using GT = GeoT<LOGN>;
  static constexpr int GRID_COL = GT::LOGA == 0 ? 1 : GT::N2 / GT::GC;
  static constexpr int GRID_ROW = GT::N1 / GT::GR;

  static cudaError_t intt_row(const ks_context *c, const u64 *src, int src_outer, u64 *dst,
                              int dst_outer, int outer, int inner, int prime_base,
                              const ulonglong2 *scale, cudaStream_t s) {
    if (outer * inner == 0) return cudaSuccess;
    const KArgs a = make_args(c);
    cudaError_t e = smem_attr(k_inv_row<LOGN>, GT::SMEM_ROW);
    if (e) return e;
    k_inv_row<LOGN><<<dim3(GRID_ROW, inner), GT::NT, GT::SMEM_ROW, s>>>(
        a, src, src_outer, dst, dst_outer, outer, prime_base, scale);
    return cudaGetLastError();
  }

  static cudaError_t intt_col(const ks_context *c, u64 *dst, int dst_outer, int outer, int inner,
                              int prime_base, const ulonglong2 *scale, cudaStream_t s) {
    if (GT::LOGA == 0 || outer * inner == 0) return cudaSuccess;
    const KArgs a = make_args(c);
    cudaError_t e = smem_attr(k_inv_col<LOGN>, GT::SMEM_COL);
    if (e) return e;
    k_inv_col<LOGN><<<dim3(GRID_COL, inner), GT::NT, GT::SMEM_COL, s>>>(a, dst, dst_outer, outer,
                                                                          prime_base, scale);
    return cudaGetLastError();
  }

  template <int PRO>
  static cudaError_t col(const ks_context *c, const TaskList &tl, const u64 *v, u64 *buf,
                         cudaStream_t s) {
    if (GT::LOGA == 0) return cudaSuccess;
    const KArgs a = make_args(c);
    cudaError_t e = smem_attr(k_fwd_col<LOGN, PRO>, GT::SMEM_COL);
    if (e) return e;
    return for_each_part(tl, [&](const TaskList &p) {
      k_fwd_col<LOGN, PRO><<<dim3(GRID_COL, p.n), GT::NT, GT::SMEM_COL, s>>>(a, p, v, buf);
    });
  }

  static cudaError_t modup_col(const ks_context *c, const TaskList &tl, const u64 *v, u64 *tmp,
                               cudaStream_t s) {
    return col<PRO_UP>(c, tl, v, tmp, s);
  }

  static cudaError_t moddown_col(const ks_context *c, const TaskList &tl, const u64 *vp,
                                 u64 *tmp2, cudaStream_t s) {
    return col<PRO_DOWN>(c, tl, vp, tmp2, s);
  }

  static cudaError_t modup_row(const ks_context *c, const TaskList &tl, int j0, int j1,
                               SlotMap sm, bool first, const u64 *d, const u64 *v,
                               const u64 *tmp, const u64 *evk, u64 *acc, cudaStream_t s) {
    if (tl.n == 0) return cudaSuccess;
    const KArgs a = make_args(c);
    constexpr int PRO = GT::LOGA == 0 ? PRO_UP : PRO_LOAD;
    cudaError_t e = smem_attr(k_fwd_row_keymult<LOGN, PRO>, GT::SMEM_ROW);
    if (e) return e;
    k_fwd_row_keymult<LOGN, PRO><<<dim3(GRID_ROW, tl.n), GT::NT, GT::SMEM_ROW, s>>>(
        a, tl, j0, j1, sm, first ? 1 : 0, d, v, tmp, evk, acc);
    return cudaGetLastError();
  }

  static cudaError_t moddown_row(const ks_context *c, const TaskList &tl, int span,
                                 const u64 *vp, const u64 *tmp2, const u64 *acc, u64 *out,
                                 cudaStream_t s) {
    const KArgs a = make_args(c);
    constexpr int PRO = GT::LOGA == 0 ? PRO_DOWN : PRO_LOAD;
    cudaError_t e = smem_attr(k_fwd_row_moddown<LOGN, PRO>, GT::SMEM_ROW);
    if (e) return e;
    return for_each_part(tl, [&](const TaskList &p) {
      k_fwd_row_moddown<LOGN, PRO><<<dim3(GRID_ROW, p.n), GT::NT, GT::SMEM_ROW, s>>>(
          a, p, span, vp, tmp2, acc, out);
    });
  }

  static cudaError_t ntt_col(const ks_context *c, const TaskList &tl, u64 *buf, cudaStream_t s) {
    return col<PRO_LOAD>(c, tl, nullptr, buf, s);
  }

  static cudaError_t ntt_row(const ks_context *c, const TaskList &tl, u64 *buf, cudaStream_t s) {
    const KArgs a = make_args(c);
    cudaError_t e = smem_attr(k_fwd_row_store<LOGN>, GT::SMEM_ROW);
    if (e) return e;
    return for_each_part(tl, [&](const TaskList &p) {
      k_fwd_row_store<LOGN><<<dim3(GRID_ROW, p.n), GT::NT, GT::SMEM_ROW, s>>>(a, p, buf);
    });
  }

  static const LaunchTable &table() {
    static const LaunchTable t = {&intt_row, &intt_col,    &modup_col, &modup_row,
                                  &moddown_col, &moddown_row, &ntt_col,  &ntt_row};
    return t;
  }
};

}  // namespace kern
}  // namespace ks
