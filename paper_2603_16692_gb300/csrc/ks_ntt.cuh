// Negacyclic NTT stages on a shared-memory tile (device side).
//
// Transform (ring x^N + 1): forward Cooley-Tukey stages s = 0..logN-1 with
// m = 2^s, t = N/2^(s+1) and twiddle psi^brv(m+i) for block i; this gives slot
// k = a(psi^(2 brv(k)+1)) (bit-reversed evaluation order). The inverse runs the
// Gentleman-Sande stages in reverse with psi^-brv(m+i), then scales by N^-1.
//
// A tile holds G independent sub-transforms of M = 2^logM points; point x of
// sub-transform g lives at s[x*P + g] (P = G+1 for G > 1: an odd pitch keeps
// 64-bit accesses free of bank conflicts when consecutive threads walk x).
// Both passes of the two-pass NTT (columns of N1 points, rows of N2 points) are
// such sub-transforms: local stage ls, local block c use the global twiddle
// index (B << ls) + c, with B = 1 for the column pass and B = N1 + row for the
// row pass. TwAcc turns (ls, c, g) into an index of the pass's twiddle table.
//
// Each round moves 2^R points of one butterfly group into registers, runs R
// stages there (radix-2^R), and writes them back.
#pragma once
#include "ks_arith.cuh"

namespace ks {

struct TwAcc {
  const ulonglong2 *tw;
  int off;        // 0: column table indexed by (1<<ls)+c;  1: row table
  int logstride;  // 0 for the column table, log N1 for the row table
  int rowbase;    // row of sub-transform g = 0 (row pass)
  int rowstep;    // 1 for the row pass, 0 for the column pass
  __device__ __forceinline__ ulonglong2 get(int ls, int c, int g) const {
    const int idx = ((((1 << ls) + c - off)) << logstride) + rowbase + g * rowstep;
    return __ldg(tw + idx);
  }
};

template <int R>
__device__ __forceinline__ void fwd_round(u64 *s, int logM, int logG, int P, int ls0,
                                          const TwAcc &tw, u64 m) {
  const u64 m2 = 2 * m;
  const int sub_log = logM - ls0 - R;
  const int ngroups = 1 << (logM - R + logG);
  const int gmask = (1 << logG) - 1;
  for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x) {
    const int g = grp & gmask;
    const int rest = grp >> logG;
    const int lo = rest & ((1 << sub_log) - 1);
    const int hi = rest >> sub_log;
    const int x0 = (hi << (logM - ls0)) + lo;
    u64 v[1 << R];
#pragma unroll
    for (int u = 0; u < (1 << R); ++u) v[u] = s[(x0 + (u << sub_log)) * P + g];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int half = 1 << (R - 1 - q);
#pragma unroll
      for (int u = 0; u < (1 << R); ++u) {
        if (u & half) continue;
        const ulonglong2 w = tw.get(ls0 + q, (hi << q) + (u >> (R - q)), g);
        u64 X = v[u];
        X = X >= m2 ? X - m2 : X;
        const u64 T = shoup(v[u + half], w.x, w.y, m);
        v[u] = X + T;
        v[u + half] = X - T + m2;
      }
    }
#pragma unroll
    for (int u = 0; u < (1 << R); ++u) s[(x0 + (u << sub_log)) * P + g] = v[u];
  }
}

template <int R>
__device__ __forceinline__ void inv_round(u64 *s, int logM, int logG, int P, int ls0,
                                          const TwAcc &tw, u64 m) {
  const u64 m2 = 2 * m;
  const int sub_log = logM - ls0 - R;
  const int ngroups = 1 << (logM - R + logG);
  const int gmask = (1 << logG) - 1;
  for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x) {
    const int g = grp & gmask;
    const int rest = grp >> logG;
    const int lo = rest & ((1 << sub_log) - 1);
    const int hi = rest >> sub_log;
    const int x0 = (hi << (logM - ls0)) + lo;
    u64 v[1 << R];
#pragma unroll
    for (int u = 0; u < (1 << R); ++u) v[u] = s[(x0 + (u << sub_log)) * P + g];
#pragma unroll
    for (int q = R - 1; q >= 0; --q) {
      const int half = 1 << (R - 1 - q);
#pragma unroll
      for (int u = 0; u < (1 << R); ++u) {
        if (u & half) continue;
        const ulonglong2 w = tw.get(ls0 + q, (hi << q) + (u >> (R - q)), g);
        const u64 X = v[u], Y = v[u + half];
        u64 S = X + Y;
        S = S >= m2 ? S - m2 : S;
        v[u] = S;
        v[u + half] = shoup(X - Y + m2, w.x, w.y, m);
      }
    }
#pragma unroll
    for (int u = 0; u < (1 << R); ++u) s[(x0 + (u << sub_log)) * P + g] = v[u];
  }
}

// Forward stages 0..logM-1 of every sub-transform in the tile. Inputs in
// [0, 4m), outputs in [0, 4m). Caller syncs before; this syncs after each round.
__device__ __forceinline__ void tile_ntt_fwd(u64 *s, int logM, int logG, int P,
                                             const TwAcc &tw, u64 m) {
  for (int ls0 = 0; ls0 < logM;) {
    const int r = min(3, logM - ls0);
    if (r == 3)
      fwd_round<3>(s, logM, logG, P, ls0, tw, m);
    else if (r == 2)
      fwd_round<2>(s, logM, logG, P, ls0, tw, m);
    else
      fwd_round<1>(s, logM, logG, P, ls0, tw, m);
    __syncthreads();
    ls0 += r;
  }
}

// Inverse stages logM-1..0. Inputs in [0, 2m), outputs in [0, 2m).
__device__ __forceinline__ void tile_ntt_inv(u64 *s, int logM, int logG, int P,
                                             const TwAcc &tw, u64 m) {
  const int nr = (logM + 2) / 3;
  for (int k = nr - 1; k >= 0; --k) {
    const int ls0 = 3 * k;
    const int r = min(3, logM - ls0);
    if (r == 3)
      inv_round<3>(s, logM, logG, P, ls0, tw, m);
    else if (r == 2)
      inv_round<2>(s, logM, logG, P, ls0, tw, m);
    else
      inv_round<1>(s, logM, logG, P, ls0, tw, m);
    __syncthreads();
  }
}

}  // namespace ks
