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

#include <algorithm>

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
  int eqp, epb;  // key layout (see ks_context)
  int tc_ap, tc_tplog;  // tensor-core basis conversion (see ks_context)
};

// Word offset of evk[j][c][limb t] (t in the context's Q u P numbering).
__host__ __device__ __forceinline__ size_t evk_off(const KArgs &a, int j, int c, int t) {
  const int tt = t < a.nq ? t : a.epb + (t - a.nq);
  return ((size_t)(j * 2 + c) * a.eqp + tt) * (size_t)a.N;
}

// The epilogue store of an output word: out = r, or r + addend (mod m).
__device__ __forceinline__ u64 out_word(const JobPtr &jp, int c, size_t idx, u64 r, u64 m) {
  if ((jp.addmask >> c) & 1) r = addmod(r, jp.add[idx], m);
  return r;
}

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
  a.eqp = c->eqp;
  a.epb = c->epb;
  a.tc_ap = c->tc_ap;
  a.tc_tplog = c->tc_tplog;
  return a;
}

// Work item y of a task descriptor (see Tasks in ks_internal.h).
__host__ __device__ __forceinline__ uint32_t decode(const KArgs &a, const Tasks &tk, int y) {
  if (tk.mode == TASK_UP) {
    for (int j = tk.j0; j < tk.j1; ++j) {
      const int lo = j * a.alpha, hi = lo + a.alpha < a.nq ? lo + a.alpha : a.nq;
      const int ovl = lo > tk.t0 ? lo : tk.t0;
      const int ovh = hi < tk.t1 ? hi : tk.t1;
      const int ov = ovh - ovl > 0 ? ovh - ovl : 0;
      const int cnt = (tk.t1 - tk.t0) - ov;
      if (y < cnt) {
        int t = tk.t0 + y;
        if (ov > 0 && t >= ovl) t += ov;
        return pack_task(t, j, j * tk.sm.sj + t * tk.sm.st + tk.sm.base);
      }
      y -= cnt;
    }
    return 0;
  }
  if (tk.mode == TASK_TARGET) return pack_task(tk.t0 + y, 0, 0);
  if (tk.mode == TASK_DOWN) {
    const int n = tk.i1 - tk.i0, c = y / n, i = tk.i0 + y % n;
    return pack_task(i, c, c * tk.span + i - tk.ibase);
  }
  if (tk.mode == TASK_DOWN1) {
    const int i = tk.i0 + y;
    return pack_task(i, 0, i - tk.ibase);
  }
  return pack_task(y % a.qp, 0, y);
}

inline int count_tasks(const ks_context *c, const Tasks &tk) {
  switch (tk.mode) {
    case TASK_UP: {
      int n = 0;
      for (int j = tk.j0; j < tk.j1; ++j) {
        const int lo = j * c->alpha, hi = std::min(lo + c->alpha, c->nq);
        const int ov = std::max(0, std::min(hi, tk.t1) - std::max(lo, tk.t0));
        n += (tk.t1 - tk.t0) - ov;
      }
      return n;
    }
    case TASK_TARGET: return tk.t1 - tk.t0;
    case TASK_DOWN: return 2 * (tk.i1 - tk.i0);
    case TASK_DOWN1: return tk.i1 - tk.i0;
    default: return tk.n;
  }
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

// load_rows that also writes the loaded words to `copy` (same layout): the input
// read from host memory leaves its device copy on the way.
template <class GT>
__device__ __forceinline__ void load_rows_copy(u64 *s, const u64 *src, u64 *copy, int r0) {
  constexpr int TILE = GT::TILE, LOGB = GT::LOGB, P = GT::PR;
  const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src + ((size_t)r0 << LOGB));
  ulonglong2 *c2 = reinterpret_cast<ulonglong2 *>(copy + ((size_t)r0 << LOGB));
#pragma unroll
  for (int it = 0; it < (TILE / 2 + GT::NT - 1) / GT::NT; ++it) {
    const int e2 = threadIdx.x + it * GT::NT;
    if ((TILE / 2) % GT::NT != 0 && e2 >= TILE / 2) break;
    const ulonglong2 val = s2[e2];
    c2[e2] = val;
    const int e = 2 * e2, g = e >> LOGB, x = e & ((1 << LOGB) - 1);
    s[x * P + g] = val.x;
    s[(x + 1) * P + g] = val.y;
  }
}

template <class GT>
__device__ __forceinline__ void store_rows(u64 *dst, const u64 *s, int r0, u64 m, u64 mu) {
  // lazy values -> canonical
  constexpr int TILE = GT::TILE, LOGB = GT::LOGB, P = GT::PR;
  ulonglong2 *d2 = reinterpret_cast<ulonglong2 *>(dst + ((size_t)r0 << LOGB));
#pragma unroll
  for (int it = 0; it < (TILE / 2 + GT::NT - 1) / GT::NT; ++it) {
    const int e2 = threadIdx.x + it * GT::NT;
    if ((TILE / 2) % GT::NT != 0 && e2 >= TILE / 2) break;
    const int e = 2 * e2, g = e >> LOGB, x = e & ((1 << LOGB) - 1);
    ulonglong2 val;
    val.x = reduce_full(s[x * P + g], m, mu);
    val.y = reduce_full(s[(x + 1) * P + g], m, mu);
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

// Stage n twiddle pairs (a contiguous slab of the table) into shared memory with one
// TMA bulk copy: thread 0 arms the CTA's barrier `bar` and issues the copy, which then
// lands while the kernel waits for its predecessor and loads its data tile. Every thread
// calls tw_ready before the first round that reads the twiddles, after a barrier that
// follows stage_tw (so the barrier's initialisation is visible).
// TMA = false (the persistent kernel, whose CTAs run many tiles): every thread copies
// its share with ordinary loads instead, and tw_ready is a no-op (the barrier before
// the first round orders the stores).
template <class GT, bool TMA = true>
__device__ __forceinline__ void stage_tw(ulonglong2 *tws, const ulonglong2 *__restrict__ src,
                                         int n, u64 *bar) {
  if (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_expect_tx(bar, (unsigned)n * 16);
      bulk_g2s(tws, src, (unsigned)n * 16, bar);
    }
  } else {
    const u64 pol = l2_keep();
    for (int k = threadIdx.x; k < n; k += GT::NT) tws[k] = ldg_pol(src + k, pol);
  }
}
// Wait for the twiddle slab; a wait that gives up records it in the context's error
// word (ks_sync_status then returns KS_ETIMEOUT) and carries on.
template <bool TMA = true>
__device__ __forceinline__ void tw_ready(u64 *bar, int *err) {
  if (TMA && !mbar_wait(bar, 0)) atomicExch(err, 1);
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
__device__ __forceinline__ void bconv_tile(u64 *s, const u64 *src, size_t N,
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
    // loads of source limb i+1 are issued before the products of limb i
    u64 x[H];
#pragma unroll
    for (int k = 0; k < H; ++k)
      x[k] = (TILE % GT::NT == 0 || threadIdx.x + (k0 + k) * GT::NT < TILE) ? src[gi[k]] : 0;
    for (int i = 0; i < nsrc; ++i) {
      const u64 c = cst[i];
      u64 xn[H];
      if (i + 1 < nsrc) {
        const u64 *sn = src + (size_t)(i + 1) * N;
#pragma unroll
        for (int k = 0; k < H; ++k)
          xn[k] = (TILE % GT::NT == 0 || threadIdx.x + (k0 + k) * GT::NT < TILE) ? sn[gi[k]] : 0;
      }
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
      if (i + 1 < nsrc) {
#pragma unroll
        for (int k = 0; k < H; ++k) x[k] = xn[k];
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
// Kernels. grid (tiles, work items, jobs); the job's pointers are js.j[blockIdx.z].

// Minimum resident blocks for a target of `threads` threads per SM (register cap).
__host__ __device__ constexpr int min_blocks(int nt, int threads) {
  return threads / nt > 0 ? threads / nt : 1;
}

// iNTT limb set `which`: 0 = the L+1 input limbs (d -> v), 1 = the P-limbs of both
// accumulators (acc -> vp). Returns (src, src_outer, dst, dst_outer, outer, prime_base,
// scale) for the current job.
struct InttSet {
  const u64 *src;
  u64 *dst;
  int src_outer, dst_outer, outer, prime_base;
  const ulonglong2 *scale;
};
__device__ __forceinline__ InttSet intt_set(const KArgs &a, const JobPtr &jp, const WsOff &o,
                                            int which) {
  InttSet r;
  if (which == 0) {
    r.src = jp.d;
    r.dst = jp.ws + o.v;
    r.src_outer = r.dst_outer = 0;
    r.outer = 1;
    r.prime_base = 0;
    r.scale = a.tab.iscale_q;
  } else {
    r.src = jp.ws + o.acc + (size_t)a.nq * a.N;
    r.dst = jp.ws + o.vp;
    r.src_outer = a.qp;
    r.dst_outer = a.np;
    r.outer = 2;
    r.prime_base = a.nq;
    r.scale = a.tab.iscale_p;
  }
  return r;
}

// Inverse NTT, row pass (global stages logN-1 .. logN1) of limb `by`: all `outer`
// polynomials in one CTA (shared twiddles), or only polynomial `only_o` when it is
// >= 0. With a single pass (N1 == 1) it also applies the per-limb scale (canonical
// output).
template <int LOGN, int RL, bool TMA = true>
__device__ __forceinline__ void inv_row_body(const KArgs &a, const JobPtr &jp, const WsOff &wo,
                                             int which, int bx, int by, unsigned char *raw,
                                             int only_o = -1) {
  using GT = GeoT<LOGN, RL, 1>;
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const InttSet is = intt_set(a, jp, wo, which);
  const int ii = by, prime = is.prime_base + ii, blk = bx;
  const int r0 = blk * GT::GR;
  const u64 m = a.tab.mod[prime].m, mu = a.tab.mod[prime].mu;
  const size_t N = a.N;
  // inverse twiddles: the forward slab of the mirrored row tile (see ks_ntt.cuh)
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, row_table<GT>(a.tab.twr_f, prime, GT::N1 / GT::GR - 1 - blk), GT::TWR,
               &twbar);
  // Reading the input from host memory (`dsrc`), this pass writes only v and the device
  // copy of d, which no kernel of the previous operation on the stream reads once its
  // last kernel runs: it starts without waiting, so its host reads overlap that kernel's
  // host writes, and waits for it at the end (keeping the chain's order for what follows).
  const bool host_in = which == 0 && jp.dsrc;
  if (!host_in) pdl_wait();
  const ulonglong2 sc = is.scale[ii];
  const int o0 = only_o < 0 ? 0 : only_o, o1 = only_o < 0 ? is.outer : only_o + 1;
  for (int o = o0; o < o1; ++o) {
    if (which == 0 && jp.dsrc)
      load_rows_copy<GT>(sm, jp.dsrc + (size_t)ii * N, const_cast<u64 *>(jp.d) + (size_t)ii * N,
                         r0);
    else
      load_rows<GT>(sm, is.src + ((size_t)o * is.src_outer + ii) * N, r0);
    __syncthreads();
    tw_ready<TMA>(&twbar, a.tab.err);
    tile_inv<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true, RL>(sm, tws, m);
    u64 *d = is.dst + ((size_t)o * is.dst_outer + ii) * N;
    if (GT::LOGA == 0) {
#pragma unroll
      for (int k = 0; k < GT::EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT != 0 && e >= GT::TILE) break;
        d[e] = csub(shoup(sm[e], sc.x, sc.y, m), m);
      }
    } else {
      store_rows<GT>(d, sm, r0, m, mu);
    }
    __syncthreads();
  }
  if (host_in) pdl_wait();
}

// Grid row of an inverse-NTT launch: the limb, and with `split` the polynomial too
// (blockIdx.y = o * limbs + limb), so that the two accumulator polynomials of the
// P-limbs run in separate CTAs when one CTA per limb would leave SMs idle.
__device__ __forceinline__ int inv_grid_row(const KArgs &a, int which, int split, int &only_o) {
  int by = blockIdx.y;
  only_o = -1;
  if (split) {
    const int inner = which == 0 ? a.nq : a.np;
    only_o = by / inner;
    by -= only_o * inner;
  }
  return by;
}

template <int LOGN, int RL>
__global__ void __launch_bounds__(GeoT<LOGN, RL, 1>::NT)
    k_inv_row(KArgs a, JobSet js, WsOff wo, int which, int split) {
  extern __shared__ __align__(16) unsigned char raw[];
  int only_o;
  const int by = inv_grid_row(a, which, split, only_o);
  inv_row_body<LOGN, RL>(a, js.j[blockIdx.z], wo, which, blockIdx.x, by, raw, only_o);
  pdl_trigger();  // the next kernel may launch once every CTA is here
}

// The bf16 bytes of a scaled column tile, in the layout of the tensor-core basis
// conversion (ks_tc.cu): the limb's columns in blocks of 2^tplog / N1 columns, block
// after block; inside a block, point (y, g) at y * (columns per block) + g, 16 bytes
// (eight bf16) per point.
template <class GT>
__device__ __forceinline__ void store_pieces(u64 *pb, const u64 *s, int c0, int tplog) {
  constexpr int TILE = GT::N1 * GT::GC;
  const int lgc = tplog - GT::LOGA;
#pragma unroll
  for (int k = 0; k < (TILE + GT::NT - 1) / GT::NT; ++k) {
    const int e = threadIdx.x + k * GT::NT;
    if (TILE % GT::NT != 0 && e >= TILE) break;
    const int y = e >> GT::LOGGC, g = e & (GT::GC - 1), col = c0 + g;
    const size_t p =
        ((size_t)(col >> lgc) << tplog) + ((size_t)y << lgc) + (col & ((1 << lgc) - 1));
    *reinterpret_cast<uint4 *>(pb + 2 * p) = bf16_bytes(s[y * GT::PC + g]);
  }
}

// Inverse NTT, column pass (global stages logN1-1 .. 0), in place, then the
// per-limb scale; `only_o` as in the row pass. pieces: write the bf16 bytes of the
// result to pv / ppv (tensor-core basis conversion) instead of the result to v / vp.
template <int LOGN, int RL, int CA, bool TMA = true>
__device__ __forceinline__ void inv_col_body(const KArgs &a, const JobPtr &jp, const WsOff &wo,
                                             int which, int bx, int by, unsigned char *raw,
                                             int only_o = -1, bool pieces = false) {
  using GT = GeoT<LOGN, RL, 0, CA>;
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, true>(raw);
  const InttSet is = intt_set(a, jp, wo, which);
  const int ii = by, prime = is.prime_base + ii;
  const int c0 = bx * GT::GC;
  const u64 m = a.tab.mod[prime].m;
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, col_table<GT>(a.tab.twc_i, prime), GT::TWC, &twbar);
  pdl_wait();
  const ulonglong2 sc = is.scale[ii];
  const int o0 = only_o < 0 ? 0 : only_o, o1 = only_o < 0 ? is.outer : only_o + 1;
  for (int o = o0; o < o1; ++o) {
    u64 *d = is.dst + ((size_t)o * is.dst_outer + ii) * (size_t)a.N;
    load_cols<GT>(sm, d, c0);
    __syncthreads();
    tw_ready<TMA>(&twbar, a.tab.err);
    tile_inv<GT::LOGA, GT::LOGGC, GT::PC, GT::NT, false, RL>(sm, tws, m);
    constexpr int TILE = GT::N1 * GT::GC;
#pragma unroll
    for (int k = 0; k < (TILE + GT::NT - 1) / GT::NT; ++k) {
      const int e = threadIdx.x + k * GT::NT;
      if (TILE % GT::NT != 0 && e >= TILE) break;
      const int y = e >> GT::LOGGC, g = e & (GT::GC - 1);
      sm[y * GT::PC + g] = csub(shoup(sm[y * GT::PC + g], sc.x, sc.y, m), m);
    }
    __syncthreads();
    if (pieces) {
      // limb ii of v, or P-limb ii of polynomial o of vp: 2N words of bytes per limb
      const size_t limb = which == 0 ? (size_t)ii : (size_t)o * a.np + ii;
      store_pieces<GT>(jp.ws + (which == 0 ? wo.pv : wo.ppv) + limb * 2 * a.N, sm, c0,
                       a.tc_tplog);
    } else {
      store_cols<GT>(d, sm, c0);
    }
    __syncthreads();
  }
}

template <int LOGN, int RL, int CA>
__global__ void __launch_bounds__(GeoT<LOGN, RL, 0, CA>::NT,
                                  min_blocks(GeoT<LOGN, RL, 0, CA>::NT, RL == 4 ? 512 : 768))
    k_inv_col(KArgs a, JobSet js, WsOff wo, int which, int split, int pieces) {
  extern __shared__ __align__(16) unsigned char raw[];
  int only_o;
  const int by = inv_grid_row(a, which, split, only_o);
  inv_col_body<LOGN, RL, CA>(a, js.j[blockIdx.z], wo, which, blockIdx.x, by, raw, only_o,
                             pieces != 0);
  pdl_trigger();  // the next kernel may launch once every CTA is here
}

// Buffers of a forward pass for job jp: the BConv sources and the output buffer.
template <int PRO>
__device__ __forceinline__ void fwd_bufs(const JobPtr &jp, const WsOff &wo, int buf,
                                         const u64 *&src, u64 *&dst) {
  if (PRO == PRO_UP) {
    src = jp.ws + wo.v;
    dst = jp.ws + wo.tmp;
  } else if (PRO == PRO_DOWN) {
    src = jp.ws + wo.vp;
    dst = jp.ws + wo.tmp2;
  } else {
    src = nullptr;
    dst = jp.ws + (buf == BUF_TMP ? wo.tmp : wo.tmp2);
  }
}

// Forward NTT, column pass (global stages 0 .. logN1-1) with a tile producer; the
// lazy ([0, 4m)) result goes to the output buffer's slot.
template <int LOGN, int RL, int PRO, int CA, bool TMA = true>
__device__ __forceinline__ void fwd_col_body(const KArgs &a, const JobPtr &jp, const WsOff &wo,
                                             const Tasks &tk, int buf, int bx, int by,
                                             unsigned char *raw, u64 *cst) {
  using GT = GeoT<LOGN, RL, 0, CA>;
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, true>(raw);
  const u64 *src;
  u64 *dst;
  fwd_bufs<PRO>(jp, wo, buf, src, dst);
  const uint32_t w = decode(a, tk, by);
  const int t = task_limb(w);
  const int c0 = bx * GT::GC;
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, col_table<GT>(a.tab.twc_f, t), GT::TWC, &twbar);
  pdl_wait();
  produce<GT, PRO, true>(a, sm, cst, w, src, dst, c0);
  __syncthreads();
  tw_ready<TMA>(&twbar, a.tab.err);
  tile_fwd<GT::LOGA, GT::LOGGC, GT::PC, GT::NT, false, RL>(sm, tws, a.tab.mod[t].m);
  store_cols<GT>(dst + (size_t)task_slot(w) * a.N, sm, c0);
}

// Tiles of 256+ threads: 4 CTAs per SM (64 registers, a few spilled words) measured
// 1-3% faster on GB300 at N >= 2^16 than the compiler's 78-register choice; smaller
// tiles keep that choice.
template <int LOGN, int RL, int PRO, int CA>
__global__ void __launch_bounds__(GeoT<LOGN, RL, 0, CA>::NT,
                                  min_blocks(GeoT<LOGN, RL, 0, CA>::NT,
                                             GeoT<LOGN, RL, 0, CA>::NT >= 256 ? 1024 : 0))
    k_fwd_col(KArgs a, JobSet js, WsOff wo, Tasks tk, int buf) {
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ u64 cst[kMaxLimbs];
  fwd_col_body<LOGN, RL, PRO, CA>(a, js.j[blockIdx.z], wo, tk, buf, blockIdx.x, blockIdx.y, raw,
                                  cst);
  pdl_trigger();  // the next kernel may launch once every CTA is here
}

// Plain forward row pass: canonical result back in place.
template <int LOGN, int RL>
__global__ void __launch_bounds__(GeoT<LOGN, RL, 1>::NT)
    k_fwd_row_store(KArgs a, JobSet js, WsOff wo, Tasks tk, int buf) {
  using GT = GeoT<LOGN, RL, 1>;
  constexpr bool TMA = true;
  extern __shared__ __align__(16) unsigned char raw[];
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const u64 *src;
  u64 *dst;
  fwd_bufs<PRO_LOAD>(js.j[blockIdx.z], wo, buf, src, dst);
  const uint32_t w = decode(a, tk, blockIdx.y);
  const int t = task_limb(w), blk = blockIdx.x, r0 = blk * GT::GR;
  const u64 m = a.tab.mod[t].m;
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, row_table<GT>(a.tab.twr_f, t, blk), GT::TWR, &twbar);
  pdl_wait();
  u64 *b = dst + (size_t)task_slot(w) * a.N;
  load_rows<GT>(sm, b, r0);
  __syncthreads();
  tw_ready<TMA>(&twbar, a.tab.err);
  tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true, RL>(sm, tws, m);
  store_rows<GT>(b, sm, r0, m, a.tab.mod[t].mu);
  pdl_trigger();  // the next kernel may launch once every CTA is here
}

// ModUp row pass fused with the key multiply. One CTA = one row tile of one
// target limb t (TASK_TARGET), over digits j0..j1-1:
//   acc_c[t] (+)= sum_j ext_j[t] * evk[j][c][t],  c = 0, 1,
// with ext_j[t] = NTT(BConv_j)[t] (Montgomery-scaled) or, on digit j's own limbs,
// the input d_t (put in Montgomery form here), so that REDC of a sum of exact
// 128-bit products is the plain sum of products mod m. The row twiddles of (t, tile)
// are staged once.
//
// The products take ext as the forward pass leaves it (below kFwdLazy * m with the
// fast butterflies; exact moduli: brought below m by two conditional subtractions),
// since REDC only needs its input below m 2^64. With at most four elements per
// thread the products of all digits are summed exactly in 128 bits and reduced once
// per output word (needs (bound of ext) * (digits) * m < 2^64, checked per CTA; the
// context guarantees digits * m < 2^64 for canonical ext); with more elements per
// thread (register budget) each product is reduced and the residues summed lazily.
template <int LOGN, int RL, int PRO, bool TMA = true>
__device__ __forceinline__ void keymult_body(const KArgs &a, const JobPtr &jp, const WsOff &wo,
                                             const Tasks &tk, int bx, int by,
                                             unsigned char *raw, u64 *cst) {
  using GT = GeoT<LOGN, RL, 1>;
  constexpr int EPT = GT::EPT;
  constexpr bool WIDE = EPT <= 4;
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const u64 *v = jp.ws + wo.v, *tmp = jp.ws + wo.tmp;
  u64 *acc = jp.ws + wo.acc;
  const int t = task_limb(decode(a, tk, by));
  const ModInfo mi = a.tab.mod[t];
  const int blk = bx, r0 = blk * GT::GR;
  const size_t N = a.N;
  const size_t off0 = (size_t)r0 << GT::LOGB;  // the tile is contiguous from here
  // One thread asks the TMA unit to pull each digit's tiles (two evk tiles and the
  // ModUp intermediate, or d on the digit's own limbs) into L2 one digit ahead.
  constexpr unsigned TB = GT::TILE * 8;
  auto prefetch_digit = [&](int j) {
    if (threadIdx.x != 0 || j >= tk.j1) return;
    prefetch_l2(jp.evk + evk_off(a, j, 0, t) + off0, TB);
    prefetch_l2(jp.evk + evk_off(a, j, 1, t) + off0, TB);
    const int lo = j * a.alpha, hi = min(lo + a.alpha, a.nq);
    if (t >= lo && t < hi)
      prefetch_l2(jp.d + (size_t)t * N + off0, TB);
    else if (GT::LOGA != 0)
      prefetch_l2(tmp + (size_t)(j * tk.sm.sj + t * tk.sm.st + tk.sm.base) * N + off0, TB);
  };
  prefetch_digit(tk.j0);
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, row_table<GT>(a.tab.twr_f, t, blk), GT::TWR, &twbar);
  pdl_wait();
  const u64 pol = l2_stream();
  const bool fast = mi.m < kFastModulus;
  // ext stays lazy when the exact digit sum of its products fits one REDC
  const int nd = tk.j1 - tk.j0;
  const bool lazy = fast && (unsigned __int128)(kFwdLazy * (WIDE ? nd : 1)) * mi.m <
                                (unsigned __int128)1 << 64;
  const u64 m2 = 2 * mi.m;
  auto ext_word = [&](u64 y) -> u64 {
    if (lazy) return y;
    if (!fast) return csub(csub(y, m2), mi.m);  // exact butterflies: below 4m
    return reduce_full(y, mi.m, mi.mu);
  };
  U128 w0[WIDE ? EPT : 1], w1[WIDE ? EPT : 1];  // exact digit sums (WIDE)
  u64 s0[WIDE ? 1 : EPT], s1[WIDE ? 1 : EPT];    // lazy residue sums in [0, 2m)
#pragma unroll
  for (int k = 0; k < (WIDE ? EPT : 1); ++k) w0[k] = w1[k] = U128{0, 0};
#pragma unroll
  for (int k = 0; k < (WIDE ? 1 : EPT); ++k) s0[k] = s1[k] = 0;
  auto mac_word = [&](int k, u64 y, const u64 *e0, const u64 *e1, int e) {
    if (WIDE) {
      mac128(w0[k], y, ldg_pol(e0 + e, pol));
      mac128(w1[k], y, ldg_pol(e1 + e, pol));
    } else {
      U128 p0 = {0, 0}, p1 = {0, 0};
      mac128(p0, y, ldg_pol(e0 + e, pol));
      mac128(p1, y, ldg_pol(e1 + e, pol));
      const u64 a0v = s0[k] + redc(p0, mi.m, mi.minv), a1v = s1[k] + redc(p1, mi.m, mi.minv);
      s0[k] = a0v >= m2 ? a0v - m2 : a0v;
      s1[k] = a1v >= m2 ? a1v - m2 : a1v;
    }
  };
  for (int j = tk.j0; j < tk.j1; ++j) {
    prefetch_digit(j + 1);
    const int lo = j * a.alpha, hi = min(lo + a.alpha, a.nq);
    const bool own = t >= lo && t < hi;
    const u64 *e0 = jp.evk + evk_off(a, j, 0, t) + off0;
    const u64 *e1 = jp.evk + evk_off(a, j, 1, t) + off0;
    if (own) {
      const u64 *dt = jp.d + (size_t)t * N + off0;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT == 0 || e < GT::TILE) {
          u64 y = shoup(__ldg(dt + e), mi.r1, mi.r1s, mi.m);  // [0, 2m)
          if (!lazy) y = csub(y, mi.m);
          mac_word(k, y, e0, e1, e);
        }
      }
    } else {
      const int slot = j * tk.sm.sj + t * tk.sm.st + tk.sm.base;
      if (GT::LOGA == 0)
        produce<GT, PRO, false>(a, sm, cst, pack_task(t, j, slot), v, tmp, r0);
      else
        produce<GT, PRO_LOAD, false>(a, sm, cst, pack_task(t, j, slot), v, tmp, r0);
      __syncthreads();
      tw_ready<TMA>(&twbar, a.tab.err);
      tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true, RL>(sm, tws, mi.m);
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT == 0 || e < GT::TILE) {
          const int g = e >> GT::LOGB, x = e & (GT::N2 - 1);
          mac_word(k, ext_word(sm[x * GT::PR + g]), e0, e1, e);
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
    u64 r0v, r1v;
    if (WIDE) {
      r0v = csub(redc(w0[k], mi.m, mi.minv), mi.m);
      r1v = csub(redc(w1[k], mi.m, mi.minv), mi.m);
    } else {
      r0v = csub(s0[k], mi.m);
      r1v = csub(s1[k], mi.m);
    }
    if (!tk.first) {
      r0v = addmod(r0v, a0[e], mi.m);
      r1v = addmod(r1v, a1[e], mi.m);
    }
    a0[e] = r0v;
    a1[e] = r1v;
  }
}

// Shared memory of the pipelined key multiply: the row twiddles, two ext tiles (odd
// pitch) and two digits' key tiles (c = 0, 1, contiguous).
template <class GT>
struct KmSmem {
  static constexpr int TW = GT::TWR * 16;
  static constexpr int TILEW = GT::N2 * GT::PR;  // words of one pitched tile
  static constexpr int KEYW = 2 * GT::TILE;      // words of one digit's two key tiles
  static constexpr int BYTES = TW + 2 * TILEW * 8 + 2 * KEYW * 8;
};

// Which row kernels (key multiply, ModDown) are pipelined: two-pass sizes with radix-4
// rounds (twice the threads per tile). With radix 8 or 16 the double buffers cost more
// occupancy than the overlap gains (measured on GB300 at (4, 2^16, 35): key multiply
// radix 4 115 -> 109 us but radix 8 119 -> 140 us; ModDown radix 4 55 -> 49 us, radix 8
// 53 -> 57 us).
template <int LOGN, int RL>
constexpr bool ROW_PIPE = geo_loga(LOGN) != 0 && RL == 2;

// The key multiply of keymult_body for N >= 2^13, software-pipelined over the digits:
// while digit j's ext tile is transformed and multiplied, the copies of digit j+1's
// tile (the ModUp intermediate, or d_t on the digit's own limbs: cp.async into the odd
// pitch) and of its two key tiles (TMA bulk copies on a barrier) are in flight into the
// other half of double buffers. Same arithmetic, same bounds and the same result as
// keymult_body.
template <int LOGN, int RL>
__device__ __forceinline__ void keymult_pipe_body(const KArgs &a, const JobPtr &jp,
                                                  const WsOff &wo, const Tasks &tk, int bx,
                                                  int by, unsigned char *raw) {
  using GT = GeoT<LOGN, RL, 1>;
  using SM = KmSmem<GT>;
  constexpr bool TMA = true;
  constexpr int EPT = GT::EPT, TILE = GT::TILE, NT = GT::NT;
  constexpr bool WIDE = EPT <= 4;
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *tiles = reinterpret_cast<u64 *>(raw + SM::TW);
  u64 *keys = tiles + 2 * SM::TILEW;
  const u64 *tmp = jp.ws + wo.tmp;
  u64 *acc = jp.ws + wo.acc;
  const int t = task_limb(decode(a, tk, by));
  const ModInfo mi = a.tab.mod[t];
  const int blk = bx, r0 = blk * GT::GR;
  const size_t N = a.N;
  const size_t off0 = (size_t)r0 << GT::LOGB;  // the tile is contiguous from here
  auto own = [&](int j) {
    const int lo = j * a.alpha;
    return t >= lo && t < min(lo + a.alpha, a.nq);
  };
  // key tiles: two contiguous TILE-word tiles per digit, one TMA bulk copy each, on the
  // buffer's barrier (use k of buffer b completes phase k & 1)
  __shared__ u64 keybar[2];
  auto issue_keys = [&](int j, int b) {
    if (threadIdx.x != 0) return;
    const u64 *e0 = jp.evk + evk_off(a, j, 0, t) + off0;
    const u64 *e1 = jp.evk + evk_off(a, j, 1, t) + off0;
    u64 *k0 = keys + b * SM::KEYW;
    mbar_expect_tx(&keybar[b], 2 * TILE * 8);
    bulk_g2s(k0, e0, TILE * 8, &keybar[b]);
    bulk_g2s(k0 + TILE, e1, TILE * 8, &keybar[b]);
  };
  auto issue_tile = [&](int j, int b) {
    const u64 *src = own(j) ? jp.d + (size_t)t * N + off0
                            : tmp + (size_t)(j * tk.sm.sj + t * tk.sm.st + tk.sm.base) * N + off0;
    u64 *st = tiles + b * SM::TILEW;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int w = threadIdx.x + k * NT;
      if (TILE % NT != 0 && w >= TILE) break;
      cp_async8(st + (w & (GT::N2 - 1)) * GT::PR + (w >> GT::LOGB), src + w);
    }
  };
  // the key tiles are inputs of the operation (no kernel of the chain writes them):
  // their first copies start before the wait for the previous kernel
  if (threadIdx.x == 0) {
    mbar_init(&keybar[0], 1);
    mbar_init(&keybar[1], 1);
  }
  issue_keys(tk.j0, 0);
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, row_table<GT>(a.tab.twr_f, t, blk), GT::TWR, &twbar);
  pdl_wait();
  issue_tile(tk.j0, 0);
  cp_async_commit();
  const bool fast = mi.m < kFastModulus;
  const int nd = tk.j1 - tk.j0;
  const bool lazy = fast && (unsigned __int128)(kFwdLazy * (WIDE ? nd : 1)) * mi.m <
                                (unsigned __int128)1 << 64;
  const u64 m2 = 2 * mi.m;
  U128 w0[WIDE ? EPT : 1], w1[WIDE ? EPT : 1];  // exact digit sums (WIDE)
  u64 s0[WIDE ? 1 : EPT], s1[WIDE ? 1 : EPT];    // lazy residue sums in [0, 2m)
#pragma unroll
  for (int k = 0; k < (WIDE ? EPT : 1); ++k) w0[k] = w1[k] = U128{0, 0};
#pragma unroll
  for (int k = 0; k < (WIDE ? 1 : EPT); ++k) s0[k] = s1[k] = 0;
  for (int j = tk.j0; j < tk.j1; ++j) {
    const int b = (j - tk.j0) & 1;
    if (j + 1 < tk.j1) {
      issue_keys(j + 1, b ^ 1);
      issue_tile(j + 1, b ^ 1);
    }
    cp_async_commit();
    cp_async_wait<1>();  // digit j's copies are done (this thread's)
    __syncthreads();     // ... and every thread's
    u64 *sm = tiles + b * SM::TILEW;
    const u64 *k0 = keys + b * SM::KEYW;
    const bool ow = own(j);
    if (!ow) {
      tw_ready<TMA>(&twbar, a.tab.err);
      tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true, RL>(sm, tws, mi.m);
    }
    if (!mbar_wait(&keybar[b], ((j - tk.j0) >> 1) & 1)) atomicExch(a.tab.err, 1);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + k * NT;
      if (TILE % NT != 0 && e >= TILE) break;
      const u64 x = sm[(e & (GT::N2 - 1)) * GT::PR + (e >> GT::LOGB)];
      u64 y;
      if (ow) {
        y = shoup(x, mi.r1, mi.r1s, mi.m);  // d_t in Montgomery form, [0, 2m)
        if (!lazy) y = csub(y, mi.m);
      } else if (lazy) {
        y = x;
      } else {
        y = fast ? reduce_full(x, mi.m, mi.mu) : csub(csub(x, m2), mi.m);
      }
      const u64 ka = k0[e], kb = k0[TILE + e];
      if (WIDE) {
        mac128(w0[k], y, ka);
        mac128(w1[k], y, kb);
      } else {
        U128 p0 = {0, 0}, p1 = {0, 0};
        mac128(p0, y, ka);
        mac128(p1, y, kb);
        const u64 a0v = s0[k] + redc(p0, mi.m, mi.minv), a1v = s1[k] + redc(p1, mi.m, mi.minv);
        s0[k] = a0v >= m2 ? a0v - m2 : a0v;
        s1[k] = a1v >= m2 ? a1v - m2 : a1v;
      }
    }
    __syncthreads();  // buffers b are free for digit j + 2
  }
  u64 *a0 = acc + (size_t)t * N + off0;
  u64 *a1 = acc + ((size_t)a.qp + t) * N + off0;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = threadIdx.x + k * NT;
    if (TILE % NT != 0 && e >= TILE) break;
    u64 r0v, r1v;
    if (WIDE) {
      r0v = csub(redc(w0[k], mi.m, mi.minv), mi.m);
      r1v = csub(redc(w1[k], mi.m, mi.minv), mi.m);
    } else {
      r0v = csub(s0[k], mi.m);
      r1v = csub(s1[k], mi.m);
    }
    if (!tk.first) {
      r0v = addmod(r0v, a0[e], mi.m);
      r1v = addmod(r1v, a1[e], mi.m);
    }
    a0[e] = r0v;
    a1[e] = r1v;
  }
}

template <int LOGN, int RL, int PRO>
__global__ void __launch_bounds__(GeoT<LOGN, RL, 1>::NT,
                                  min_blocks(GeoT<LOGN, RL, 1>::NT,
                                             RL == 4 ? 384 : RL == 2 ? 1024 : 768))
    k_fwd_row_keymult(KArgs a, JobSet js, WsOff wo, Tasks tk) {
  extern __shared__ __align__(16) unsigned char raw[];
  // Targets in reverse: the P-limb targets, listed last, have no digit of their own (one
  // more NTT per CTA), so starting them first shortens the tail of multi-wave launches
  // (measured on GB300 at (4, 2^16, 35): 125 -> 121 us for this launch).
  const int by = gridDim.y - 1 - blockIdx.y;
  if constexpr (ROW_PIPE<LOGN, RL>) {
    keymult_pipe_body<LOGN, RL>(a, js.j[blockIdx.z], wo, tk, blockIdx.x, by, raw);
  } else {
    __shared__ u64 cst[GeoT<LOGN, RL, 1>::LOGA == 0 ? kMaxLimbs : 1];
    keymult_body<LOGN, RL, PRO>(a, js.j[blockIdx.z], wo, tk, blockIdx.x, by, raw, cst);
  }
  pdl_trigger();  // the next kernel may launch once every CTA is here
}

// ModDown row pass fused with the final scaling, both polynomials c = 0, 1 of
// limb i (TASK_DOWN1) in one CTA (shared twiddles):
//   out_c[i] = (acc_c[i] - NTT(BConv_{P->Q}(c))[i]) * P^-1 mod q_i.
template <int LOGN, int RL, int PRO, bool TMA = true>
__device__ __forceinline__ void moddown_body(const KArgs &a, const JobPtr &jp, const WsOff &wo,
                                             const Tasks &tk, int bx, int by,
                                             unsigned char *raw, u64 *cst) {
  using GT = GeoT<LOGN, RL, 1>;
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *sm = tile_ptr<GT, false>(raw);
  const u64 *vp = jp.ws + wo.vp, *tmp2 = jp.ws + wo.tmp2, *acc = jp.ws + wo.acc;
  const uint32_t w = decode(a, tk, by);
  const int i = task_limb(w), blk = bx, r0 = blk * GT::GR;
  const u64 m = a.tab.mod[i].m;
  const ulonglong2 pv = a.tab.pinv[i];
  const size_t N = a.N;
  const size_t off0 = (size_t)r0 << GT::LOGB;
  // The NTT output z enters the scaling lazy: below kFwdLazy * m (fast butterflies) or,
  // after one conditional subtraction, below 2m (exact); acc + zb - z is then positive
  // and below (kFwdLazy + 1) m < 2^64, and the Shoup product by P^-1 takes any word.
  const bool fast = m < kFastModulus;
  const u64 m2 = 2 * m, zb = fast ? kFwdLazy * m : m2;
  if (threadIdx.x == 0)
    for (int c = 0; c < 2; ++c) prefetch_l2(acc + ((size_t)c * a.qp + i) * N + off0, GT::TILE * 8);
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, row_table<GT>(a.tab.twr_f, i, blk), GT::TWR, &twbar);
  pdl_wait();
  for (int c = 0; c < 2; ++c) {
    const uint32_t wc = pack_task(i, c, task_slot(w) + c * tk.span);
    if (GT::LOGA == 0)
      produce<GT, PRO, false>(a, sm, cst, wc, vp, tmp2, r0);
    else
      produce<GT, PRO_LOAD, false>(a, sm, cst, wc, vp, tmp2, r0);
    __syncthreads();
    tw_ready<TMA>(&twbar, a.tab.err);
    tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true, RL>(sm, tws, m);
    const u64 *ac = acc + ((size_t)c * a.qp + i) * N + off0;
    const size_t ob = ((size_t)c * a.nq + i) * N + off0;
    u64 *o = jp.out + ob;
    if ((jp.addmask >> c) & 1) {
      const u64 *ad = jp.add + ob;
#pragma unroll
      for (int k = 0; k < GT::EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT != 0 && e >= GT::TILE) break;
        const int g = e >> GT::LOGB, x = e & (GT::N2 - 1);
        const u64 z = fast ? sm[x * GT::PR + g] : csub(sm[x * GT::PR + g], m2);
        o[e] = addmod(csub(shoup(ac[e] + zb - z, pv.x, pv.y, m), m), ad[e], m);
      }
    } else {
#pragma unroll
      for (int k = 0; k < GT::EPT; ++k) {
        const int e = threadIdx.x + k * GT::NT;
        if (GT::TILE % GT::NT != 0 && e >= GT::TILE) break;
        const int g = e >> GT::LOGB, x = e & (GT::N2 - 1);
        const u64 z = fast ? sm[x * GT::PR + g] : csub(sm[x * GT::PR + g], m2);
        o[e] = csub(shoup(ac[e] + zb - z, pv.x, pv.y, m), m);
      }
    }
    __syncthreads();
  }
}

// Shared memory of the pipelined ModDown row pass: the row twiddles, the two
// polynomials' NTT tiles (odd pitch) and their accumulator tiles (contiguous).
template <class GT>
struct MdSmem {
  static constexpr int TW = GT::TWR * 16;
  static constexpr int TILEW = GT::N2 * GT::PR;
  static constexpr int BYTES = TW + 2 * TILEW * 8 + 2 * GT::TILE * 8;
};

// moddown_body for N >= 2^13 with both polynomials' input tiles (cp.async into the odd
// pitch) and accumulator tiles (TMA bulk copies on a barrier) copied into shared memory
// at the start: the copies of c = 1 and of the accumulators are in flight while c = 0
// is transformed. Same arithmetic and result.
template <int LOGN, int RL>
__device__ __forceinline__ void moddown_pipe_body(const KArgs &a, const JobPtr &jp,
                                                  const WsOff &wo, const Tasks &tk, int bx,
                                                  int by, unsigned char *raw) {
  using GT = GeoT<LOGN, RL, 1>;
  using SM = MdSmem<GT>;
  constexpr bool TMA = true;
  constexpr int EPT = GT::EPT, TILE = GT::TILE, NT = GT::NT;
  ulonglong2 *tws = reinterpret_cast<ulonglong2 *>(raw);
  u64 *tiles = reinterpret_cast<u64 *>(raw + SM::TW);
  u64 *accs = tiles + 2 * SM::TILEW;
  const u64 *tmp2 = jp.ws + wo.tmp2, *acc = jp.ws + wo.acc;
  const uint32_t w = decode(a, tk, by);
  const int i = task_limb(w), blk = bx, r0 = blk * GT::GR;
  const u64 m = a.tab.mod[i].m;
  const ulonglong2 pv = a.tab.pinv[i];
  const size_t N = a.N;
  const size_t off0 = (size_t)r0 << GT::LOGB;
  // the NTT output enters the scaling lazy, as in moddown_body
  const bool fast = m < kFastModulus;
  const u64 m2 = 2 * m, zb = fast ? kFwdLazy * m : m2;
  __shared__ u64 twbar;
  stage_tw<GT, TMA>(tws, row_table<GT>(a.tab.twr_f, i, blk), GT::TWR, &twbar);
  pdl_wait();
  // the accumulator tiles (contiguous): one TMA bulk copy each, on one barrier
  __shared__ u64 accbar;
  if (threadIdx.x == 0) {
    mbar_init(&accbar, 1);
    mbar_expect_tx(&accbar, 2 * TILE * 8);
    for (int c = 0; c < 2; ++c)
      bulk_g2s(accs + c * TILE, acc + ((size_t)c * a.qp + i) * N + off0, TILE * 8, &accbar);
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const u64 *src = tmp2 + (size_t)(task_slot(w) + c * tk.span) * N + off0;
    u64 *st = tiles + c * SM::TILEW;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + k * NT;
      if (TILE % NT != 0 && e >= TILE) break;
      cp_async8(st + (e & (GT::N2 - 1)) * GT::PR + (e >> GT::LOGB), src + e);
    }
    cp_async_commit();
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (c == 0)
      cp_async_wait<1>();
    else
      cp_async_wait<0>();
    __syncthreads();
    u64 *sm = tiles + c * SM::TILEW;
    const u64 *sa = accs + c * TILE;
    tw_ready<TMA>(&twbar, a.tab.err);
    tile_fwd<GT::LOGB, GT::LOGGR, GT::PR, GT::NT, true, RL>(sm, tws, m);
    if (c == 0 && !mbar_wait(&accbar, 0)) atomicExch(a.tab.err, 1);
    const size_t ob = ((size_t)c * a.nq + i) * N + off0;
    u64 *o = jp.out + ob;
    const bool add = (jp.addmask >> c) & 1;
    const u64 *ad = jp.add + ob;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + k * NT;
      if (TILE % NT != 0 && e >= TILE) break;
      const u64 zr = sm[(e & (GT::N2 - 1)) * GT::PR + (e >> GT::LOGB)];
      const u64 z = fast ? zr : csub(zr, m2);
      u64 r = csub(shoup(sa[e] + zb - z, pv.x, pv.y, m), m);
      if (add) r = addmod(r, ad[e], m);
      o[e] = r;
    }
  }
}

template <int LOGN, int RL, int PRO>
__global__ void __launch_bounds__(GeoT<LOGN, RL, 1>::NT,
                                  min_blocks(GeoT<LOGN, RL, 1>::NT, RL == 4 ? 0 : 1024))
    k_fwd_row_moddown(KArgs a, JobSet js, WsOff wo, Tasks tk) {
  extern __shared__ __align__(16) unsigned char raw[];
  // host-buffer operation: let the next one's input pass (which reads host memory and
  // does not wait for this kernel before it ends) start while this one writes its result
  // to host memory
  if (js.j[blockIdx.z].dsrc) pdl_trigger();
  if constexpr (ROW_PIPE<LOGN, RL>) {
    moddown_pipe_body<LOGN, RL>(a, js.j[blockIdx.z], wo, tk, blockIdx.x, blockIdx.y, raw);
  } else {
    __shared__ u64 cst[GeoT<LOGN, RL, 1>::LOGA == 0 ? kMaxLimbs : 1];
    moddown_body<LOGN, RL, PRO>(a, js.j[blockIdx.z], wo, tk, blockIdx.x, blockIdx.y, raw, cst);
  }
  pdl_trigger();  // the next kernel may launch once every CTA is here
}

// ---------------------------------------------------------------------------
// Launchers for one N and radix.

cudaError_t smem_opt_in(const void *kernel, int bytes);

template <class K>
inline cudaError_t smem_attr(K kernel, int bytes) {
  return smem_opt_in(reinterpret_cast<const void *>(kernel), bytes);
}

inline KArgs args_of(const ks_context *c) { return make_args(c); }

// Below four CTAs per SM of a GB300 (152 SMs) a launch is latency-bound on its few
// CTAs' serial work (measured at (2, 2^15, 10): the accumulator iNTT passes 12.1 ->
// 10.1 us and 12.0 -> 10.8 us with one CTA per polynomial).
constexpr int kSplitCtas = 4 * 152;

template <int LOGN, int RL, int CA = 0>
struct Launch {
  using GTC = GeoT<LOGN, RL, 0, CA>;  // column-pass geometry (CA: alternative tile)
  using GTR = GeoT<LOGN, RL, 1>;  // row-pass geometry
  static constexpr int GRID_COL = GTC::LOGA == 0 ? 1 : GTC::N2 / GTC::GC;
  static constexpr int GRID_ROW = GTR::N1 / GTR::GR;
  static constexpr int PRO_ROW_UP = GTR::LOGA == 0 ? PRO_UP : PRO_LOAD;
  static constexpr int PRO_ROW_DOWN = GTR::LOGA == 0 ? PRO_DOWN : PRO_LOAD;
  // the pipelined row kernels reserve their double buffers
  static constexpr int SMEM_KM = ROW_PIPE<LOGN, RL> ? KmSmem<GTR>::BYTES : GTR::SMEM_ROW;
  static constexpr int SMEM_MD = ROW_PIPE<LOGN, RL> ? MdSmem<GTR>::BYTES : GTR::SMEM_ROW;

  static cudaError_t prepare() {
    cudaError_t e;
    if ((e = smem_attr(k_inv_row<LOGN, RL>, GTR::SMEM_ROW))) return e;
    if ((e = smem_attr(k_fwd_row_store<LOGN, RL>, GTR::SMEM_ROW))) return e;
    if ((e = smem_attr(k_fwd_row_keymult<LOGN, RL, PRO_ROW_UP>, SMEM_KM))) return e;
    if ((e = smem_attr(k_fwd_row_moddown<LOGN, RL, PRO_ROW_DOWN>, SMEM_MD))) return e;
    if (GTC::LOGA > 0) {
      if ((e = smem_attr(k_inv_col<LOGN, RL, CA>, GTC::SMEM_COL))) return e;
      if ((e = smem_attr(k_fwd_col<LOGN, RL, PRO_LOAD, CA>, GTC::SMEM_COL))) return e;
      if ((e = smem_attr(k_fwd_col<LOGN, RL, PRO_UP, CA>, GTC::SMEM_COL))) return e;
      if ((e = smem_attr(k_fwd_col<LOGN, RL, PRO_DOWN, CA>, GTC::SMEM_COL))) return e;
    }
    return cudaSuccess;
  }

  static int count(const ks_context *c, const Tasks &tk) { return count_tasks(c, tk); }

  // The accumulator P-limbs (which = 1) hold two polynomials per limb: they get one CTA
  // each when a CTA per limb would give fewer than kSplitCtas CTAs.
  static int inv_split(int grid, int inner, int which, int jobs) {
    return which == 1 && grid * inner * jobs < kSplitCtas ? 1 : 0;
  }

  static cudaError_t intt_row(const ks_context *c, const JobSet &js, const WsOff &wo, int which,
                              cudaStream_t s) {
    const int inner = which == 0 ? c->nq : c->np;
    if (inner == 0 || js.n == 0) return cudaSuccess;
    const int split = inv_split(GRID_ROW, inner, which, js.n);
    return launch_pdl(k_inv_row<LOGN, RL>, dim3(GRID_ROW, inner << split, js.n), dim3(GTR::NT),
                      GTR::SMEM_ROW, s, args_of(c), js, wo, which, split);
  }

  static cudaError_t intt_col_p(const ks_context *c, const JobSet &js, const WsOff &wo,
                                int which, int pieces, cudaStream_t s) {
    const int inner = which == 0 ? c->nq : c->np;
    if (GTC::LOGA == 0 || inner == 0 || js.n == 0) return cudaSuccess;
    const int split = inv_split(GRID_COL, inner, which, js.n);
    return launch_pdl(k_inv_col<LOGN, RL, CA>, dim3(GRID_COL, inner << split, js.n), dim3(GTC::NT),
                      GTC::SMEM_COL, s, args_of(c), js, wo, which, split, pieces);
  }
  static cudaError_t intt_col(const ks_context *c, const JobSet &js, const WsOff &wo, int which,
                              cudaStream_t s) {
    return intt_col_p(c, js, wo, which, 0, s);
  }
  static cudaError_t intt_col_tc(const ks_context *c, const JobSet &js, const WsOff &wo,
                                 int which, cudaStream_t s) {
    return intt_col_p(c, js, wo, which, 1, s);
  }

  template <int PRO>
  static cudaError_t col(const ks_context *c, const JobSet &js, const WsOff &wo,
                         const Tasks &tk, int buf, cudaStream_t s) {
    const int n = count_tasks(c, tk);
    if (GTC::LOGA == 0 || n == 0 || js.n == 0) return cudaSuccess;
    return launch_pdl(k_fwd_col<LOGN, RL, PRO, CA>, dim3(GRID_COL, n, js.n), dim3(GTC::NT),
                      GTC::SMEM_COL, s, args_of(c), js, wo, tk, buf);
  }

  static cudaError_t modup_col(const ks_context *c, const JobSet &js, const WsOff &wo,
                               const Tasks &tk, cudaStream_t s) {
    return col<PRO_UP>(c, js, wo, tk, BUF_TMP, s);
  }

  static cudaError_t moddown_col(const ks_context *c, const JobSet &js, const WsOff &wo,
                                 const Tasks &tk, cudaStream_t s) {
    return col<PRO_DOWN>(c, js, wo, tk, BUF_TMP2, s);
  }

  static cudaError_t modup_row(const ks_context *c, const JobSet &js, const WsOff &wo,
                               const Tasks &tk, cudaStream_t s) {
    const int n = count_tasks(c, tk);
    if (n == 0 || js.n == 0) return cudaSuccess;
    return launch_pdl(k_fwd_row_keymult<LOGN, RL, PRO_ROW_UP>, dim3(GRID_ROW, n, js.n),
                      dim3(GTR::NT), SMEM_KM, s, args_of(c), js, wo, tk);
  }

  static cudaError_t moddown_row(const ks_context *c, const JobSet &js, const WsOff &wo,
                                 const Tasks &tk, cudaStream_t s) {
    const int n = count_tasks(c, tk);
    if (n == 0 || js.n == 0) return cudaSuccess;
    return launch_pdl(k_fwd_row_moddown<LOGN, RL, PRO_ROW_DOWN>, dim3(GRID_ROW, n, js.n),
                      dim3(GTR::NT), SMEM_MD, s, args_of(c), js, wo, tk);
  }

  static cudaError_t ntt_col(const ks_context *c, const JobSet &js, const WsOff &wo,
                             const Tasks &tk, int buf, cudaStream_t s) {
    return col<PRO_LOAD>(c, js, wo, tk, buf, s);
  }

  static cudaError_t ntt_row(const ks_context *c, const JobSet &js, const WsOff &wo,
                             const Tasks &tk, int buf, cudaStream_t s) {
    const int n = count_tasks(c, tk);
    if (n == 0 || js.n == 0) return cudaSuccess;
    return launch_pdl(k_fwd_row_store<LOGN, RL>, dim3(GRID_ROW, n, js.n), dim3(GTR::NT),
                      GTR::SMEM_ROW, s, args_of(c), js, wo, tk, buf);
  }

  static const LaunchTable &table() {
    static const LaunchTable t = {&prepare,     &count,       &intt_row,  &intt_col,
                                  &intt_col_tc, &modup_col,   &modup_row, &moddown_col,
                                  &moddown_row, &ntt_col,     &ntt_row};
    return t;
  }
};

}  // namespace kern
}  // namespace ks
