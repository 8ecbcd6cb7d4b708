// Negacyclic NTT stages on a shared-memory tile (device side), with the tile
// geometry fixed at compile time.
//
// Transform (ring x^N + 1): forward Cooley-Tukey stages s = 0..logN-1 with
// m = 2^s, t = N/2^(s+1) and twiddle psi^brv(m+i) for block i; this gives slot
// k = a(psi^(2 brv(k)+1)) (bit-reversed evaluation order). The inverse runs the
// Gentleman-Sande stages in reverse with psi^-brv(m+i), then scales by N^-1.
//
// The inverse twiddle of block i at stage s is psi^-brv(2^s + i) = -psi^brv(2^s + i'),
// with i' = i XOR (2^s - 1) (psi^N = -1, and brv maps the complement of i to N minus
// the exponent). The inverse row pass therefore reads the forward row table: the slab
// of the mirrored row tile, mirrored inside (row g -> G-1-g, block c -> 2^ls-1-c),
// and its Gentleman-Sande butterflies take (Y - X) w instead of (X - Y)(-w).
//
// N = N1 * N2. The column pass runs stages 0..log N1-1 on the N2 columns (each an
// N1-point transform with twiddle index 2^ls + c for local stage ls, block c);
// the row pass runs the remaining stages on the N1 rows of N2 contiguous points
// (twiddle index (N1 + row) 2^ls + c). For N <= 4096 one row pass does all.
//
// A tile holds G = 2^LOGG sub-transforms of M = 2^LOGM points; point x of
// sub-transform g lives at s[x*P + g] (P = G+1 for G > 1: an odd pitch keeps
// 64-bit accesses free of bank conflicts). Twiddles sit in shared memory:
// column pass: tw[k], k = 2^ls + c (the first N1 entries of the table);
// row pass: tw[(2^ls - 1 + c) * G + g] (the tile's rows, stage-major).
//
// Each round moves 2^R points of one butterfly group into registers, runs R
// stages there (radix-2^R), and writes them back; every offset is a constant.
#pragma once
#include "ks_arith.cuh"
#include "ks_internal.h"

namespace ks {

// Compile-time geometry of the two passes for N = 2^LOGN (also used on the host
// to lay out the row-pass twiddle table by row tile).
__host__ __device__ constexpr int geo_loga(int logn) { return logn <= 12 ? 0 : logn / 2; }
// Tiles (measured on GB300). Column pass: 2^10 points up to N = 2^15, 2^11 above (at
// 2^15 the smaller tiles double the CTAs of the one-wave launches, 94.8 -> 85.8 us per
// KeySwitch at (2, 2^15, 10); at 2^16 the column passes are slower with 2^10 points).
// Row pass: 2^9 points up to N = 2^15, 2^10 above (2^9 against 2^10: 36.9 -> 33.3 us at
// (2, 2^13, 7), 81.5 -> 77.8 us at (2, 2^14, 20), 13.4 k -> 14.0 k KeySwitch/s at
// (2, 2^15, 10); at (4, 2^16, 35) 2^9 is 2% slower).
__host__ __device__ constexpr int geo_tile_log_col(int logn) {
  return logn <= 12 ? logn : (logn >= 16 ? 11 : 10);
}
// The alternative column tile the tuner may pick (CA = 1): the other of 2^10 / 2^11.
__host__ __device__ constexpr int geo_tile_log_col_alt(int logn) {
  return logn <= 12 ? logn : (logn >= 16 ? 10 : 11);
}
__host__ __device__ constexpr int geo_tile_log_row(int logn) {
  return logn <= 12 ? logn : (logn <= 15 ? 9 : 10);
}
__host__ __device__ constexpr int geo_loggr(int logn) {
  return geo_tile_log_row(logn) - (logn - geo_loga(logn));
}

// RL: log2 of the radix of the register rounds; a thread holds 2^RL points.
// ROW: geometry of the row pass (1) or of the column pass (0); a kernel runs one pass
// and uses only that pass's fields. CA: the column pass uses the alternative tile.
template <int LOGN, int RL_, int ROW, int CA = 0>
struct GeoT {
  static constexpr int RL = RL_;
  static constexpr int LOGA = geo_loga(LOGN);  // log N1
  static constexpr int LOGB = LOGN - LOGA;     // log N2
  static constexpr int TILE_LOG =
      ROW ? geo_tile_log_row(LOGN) : (CA ? geo_tile_log_col_alt(LOGN) : geo_tile_log_col(LOGN));
  static constexpr int LOGGC = LOGA == 0 ? 0 : TILE_LOG - LOGA;  // columns per column tile
  static constexpr int LOGGR = TILE_LOG - LOGB;                  // rows per row tile
  static constexpr int TILE = 1 << TILE_LOG;
  static constexpr int NT = (TILE >> RL) < 32 ? 32 : (TILE >> RL);  // one group per thread
  static constexpr int EPT = (TILE + NT - 1) / NT;           // tile elements per thread
  static constexpr int GC = 1 << LOGGC, GR = 1 << LOGGR;
  static constexpr int PC = GC == 1 ? 1 : GC + 1;
  static constexpr int PR = GR == 1 ? 1 : GR + 1;
  static constexpr int N1 = 1 << LOGA, N2 = 1 << LOGB;
  static constexpr int TWC = N1;                  // column-pass twiddles per tile
  static constexpr int TWR = (N2 - 1) * GR;       // row-pass twiddles per tile
  static constexpr int SMEM_COL = (N1 * PC) * 8 + TWC * 16;
  static constexpr int SMEM_ROW = (N2 * PR) * 8 + TWR * 16;
};

__device__ __forceinline__ void bfly_fwd(u64 &a, u64 &b, const ulonglong2 w, u64 m, u64 m2) {
  u64 X = a;
  X = X >= m2 ? X - m2 : X;
  const u64 T = shoup(b, w.x, w.y, m);
  a = X + T;
  b = X - T + m2;
}

__device__ __forceinline__ void bfly_inv(u64 &a, u64 &b, const ulonglong2 w, u64 m, u64 m2) {
  const u64 X = a, Y = b;
  u64 S = X + Y;
  a = S >= m2 ? S - m2 : S;
  b = shoup(X - Y + m2, w.x, w.y, m);
}

// Fast butterflies for m < kFastModulus (2^51). Forward: no reduction of the
// upper input, approximate Shoup product T in [0, 4m): each stage raises the
// bound by 4m, so a column pass (<= 8 stages) starting below 2m ends below 34m
// and the row pass (<= 9 stages) below 70m (12 single-pass stages: below 50m).
__device__ __forceinline__ void bfly_fwd_fast(u64 &a, u64 &b, const ulonglong2 w, u64 m,
                                              u64 m4) {
  const u64 X = a;
  const u64 T = shoup4(b, w.x, w.y, m);
  a = X + T;
  b = X - T + m4;
}
// Inverse: canonical inputs; the k-th processed stage adds without reduction and
// biases the difference by B_k = m 2^(k+1) (>= the bound of both inputs); the
// product is taken with the approximate quotient, in [0, 4m). After K stages all
// values are below m 2^(K+1) <= 2^13 m < 2^64.
__device__ __forceinline__ void bfly_inv_fast(u64 &a, u64 &b, const ulonglong2 w, u64 m,
                                              u64 bias) {
  const u64 X = a, Y = b;
  a = X + Y;
  b = shoup4(X - Y + bias, w.x, w.y, m);
}
// The same two butterflies with the negated twiddle -w given as w (mirrored tables).
__device__ __forceinline__ void bfly_inv_neg(u64 &a, u64 &b, const ulonglong2 w, u64 m,
                                             u64 m2) {
  const u64 X = a, Y = b;
  u64 S = X + Y;
  a = S >= m2 ? S - m2 : S;
  b = shoup(Y - X + m2, w.x, w.y, m);
}
__device__ __forceinline__ void bfly_inv_fast_neg(u64 &a, u64 &b, const ulonglong2 w, u64 m,
                                                  u64 bias) {
  const u64 X = a, Y = b;
  a = X + Y;
  b = shoup4(Y - X + bias, w.x, w.y, m);
}

// SPLIT: the block runs several tiles side by side, NT threads each (NT a power of
// two); a thread works on the tile of its group of NT (the caller picks s, tw, m).
template <int LOGM, int LOGG, int P, int NT, bool ROW, bool INV, int LS0, int R, bool FAST,
          bool SPLIT = false>
__device__ __forceinline__ void ntt_round(u64 *s, const ulonglong2 *tw, u64 m) {
  constexpr int SUB = LOGM - LS0 - R;
  constexpr int NG = 1 << (LOGM - R + LOGG);
  const u64 m2 = 2 * m, m4 = 4 * m;
  const int tid = SPLIT ? (int)(threadIdx.x & (NT - 1)) : (int)threadIdx.x;
#pragma unroll
  for (int it = 0; it < (NG + NT - 1) / NT; ++it) {
    const int grp = tid + it * NT;
    if (NG % NT != 0 && grp >= NG) break;
    const int g = grp & ((1 << LOGG) - 1);
    const int rest = grp >> LOGG;
    const int lo = rest & ((1 << SUB) - 1);
    const int hi = rest >> SUB;
    u64 *base = s + ((hi << (LOGM - LS0)) + lo) * P + g;
    u64 v[1 << R];
#pragma unroll
    for (int u = 0; u < (1 << R); ++u) v[u] = base[(u << SUB) * P];
    if (!INV) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int half = 1 << (R - 1 - q);
        // twiddle index of local stage LS0+q, block (hi << q) + (u >> (R-q))
        const ulonglong2 *twq =
            ROW ? tw + ((((1 << (LS0 + q)) - 1 + (hi << q)) << LOGG) + g)
                : tw + (1 << (LS0 + q)) + (hi << q);
#pragma unroll
        for (int u = 0; u < (1 << R); ++u) {
          if (u & half) continue;
          const ulonglong2 w = twq[ROW ? ((u >> (R - q)) << LOGG) : (u >> (R - q))];
          if (FAST)
            bfly_fwd_fast(v[u], v[u + half], w, m, m4);
          else
            bfly_fwd(v[u], v[u + half], w, m, m2);
        }
      }
    } else {
#pragma unroll
      for (int q = R - 1; q >= 0; --q) {
        const int half = 1 << (R - 1 - q);
        // row pass: the forward slab of the mirrored tile, entry (2^ls - 1 + c') G + g'
        // with c' = 2^ls - 1 - c, g' = G - 1 - g (negated twiddles)
        const ulonglong2 *twq =
            ROW ? tw + ((((2 << (LS0 + q)) - 2 - (hi << q)) << LOGG) + ((1 << LOGG) - 1 - g))
                : tw + (1 << (LS0 + q)) + (hi << q);
        // processed-stage index k = LOGM-1-ls, bias m 2^(k+1)
        const u64 bias = m << (LOGM - (LS0 + q));
#pragma unroll
        for (int u = 0; u < (1 << R); ++u) {
          if (u & half) continue;
          if (ROW) {
            const ulonglong2 w = twq[-((u >> (R - q)) << LOGG)];
            if (FAST)
              bfly_inv_fast_neg(v[u], v[u + half], w, m, bias);
            else
              bfly_inv_neg(v[u], v[u + half], w, m, m2);
          } else {
            const ulonglong2 w = twq[u >> (R - q)];
            if (FAST)
              bfly_inv_fast(v[u], v[u + half], w, m, bias);
            else
              bfly_inv(v[u], v[u + half], w, m, m2);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < (1 << R); ++u) base[(u << SUB) * P] = v[u];
  }
}

// Forward stages 0..LOGM-1 of every sub-transform in the tile, in rounds of at
// most RM stages. Inputs in [0, 4m), outputs in [0, 4m). Caller syncs before;
// each round syncs after.
// Barrier after a round: the whole block (BARN = 0), or named barrier `id` over BARN
// threads (a group of the block; the others run another role or another group).
template <int BARN>
__device__ __forceinline__ void round_sync(int id = 1) {
  if constexpr (BARN == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(BARN) : "memory");
}

template <int LOGM, int LOGG, int P, int NT, bool ROW, int RM, bool FAST, int LS0 = 0,
          bool SPLIT = false, int BARN = 0>
__device__ __forceinline__ void tile_fwd_t(u64 *s, const ulonglong2 *tw, u64 m, int bar_id = 1) {
  if constexpr (LS0 < LOGM) {
    constexpr int R = (LOGM - LS0) >= RM ? RM : (LOGM - LS0);
    ntt_round<LOGM, LOGG, P, NT, ROW, false, LS0, R, FAST, SPLIT>(s, tw, m);
    round_sync<BARN>(bar_id);
    tile_fwd_t<LOGM, LOGG, P, NT, ROW, RM, FAST, LS0 + R, SPLIT, BARN>(s, tw, m, bar_id);
  }
}

// Bound of the lazy forward outputs with the fast butterflies: every forward pass
// (column then row, or one single pass) of the library ends below kFwdLazy * m.
constexpr u64 kFwdLazy = 70;

// Forward stages on the tile; fast butterflies when m < kFastModulus. Outputs are
// lazy (below kFwdLazy * m fast, 4m exact): reduce before use, or feed them to a
// reduction whose input bound allows it.
template <int LOGM, int LOGG, int P, int NT, bool ROW, int RM = 3>
__device__ __forceinline__ void tile_fwd(u64 *s, const ulonglong2 *tw, u64 m) {
  if (m < kFastModulus)
    tile_fwd_t<LOGM, LOGG, P, NT, ROW, RM, true>(s, tw, m);
  else
    tile_fwd_t<LOGM, LOGG, P, NT, ROW, RM, false>(s, tw, m);
}

// Inverse stages LOGM-1..0. Inputs in [0, 2m), outputs in [0, 2m).
template <int LOGM, int LOGG, int P, int NT, bool ROW, int RM, bool FAST,
          int K = (LOGM + RM - 1) / RM - 1>
__device__ __forceinline__ void tile_inv_t(u64 *s, const ulonglong2 *tw, u64 m) {
  if constexpr (K >= 0 && LOGM > 0) {
    constexpr int LS0 = RM * K;
    constexpr int R = (LOGM - LS0) >= RM ? RM : (LOGM - LS0);
    ntt_round<LOGM, LOGG, P, NT, ROW, true, LS0, R, FAST>(s, tw, m);
    __syncthreads();
    tile_inv_t<LOGM, LOGG, P, NT, ROW, RM, FAST, K - 1>(s, tw, m);
  }
}

// Inverse stages; inputs canonical (fast) or below 2m (exact). Outputs lazy (below
// 2^13 m fast, 2m exact): reduce with reduce_full or a Shoup scaling before use.
template <int LOGM, int LOGG, int P, int NT, bool ROW, int RM = 3>
__device__ __forceinline__ void tile_inv(u64 *s, const ulonglong2 *tw, u64 m) {
  if (m < kFastModulus)
    tile_inv_t<LOGM, LOGG, P, NT, ROW, RM, true>(s, tw, m);
  else
    tile_inv_t<LOGM, LOGG, P, NT, ROW, RM, false>(s, tw, m);
}

}  // namespace ks
