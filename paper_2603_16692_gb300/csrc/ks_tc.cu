// Fast basis conversion (the ModUp and ModDown BConv of Sec. II-A) on the tensor cores
// (tcgen05, sm_103a), fused with the first forward NTT pass.
//
// The conversion of one column tile is an integer matrix product,
//   S[p][t] = sum_i x_i[p] * c_i[t]    (x_i < 2^62 source residues, c_i < 2^62 constants),
// that must be exact (128 bits) before its one Montgomery reduction. It runs on the
// bf16 tensor cores exactly by splitting both operands into bytes:
//   x_i = sum_a x_ia 2^(8a),  c_i = sum_b c_ib 2^(8b)   (a, b = 0..7),
//   S = sum_s v_s 2^(8s),  v_s = sum_i sum_{a+b=s} x_ia c_ib   (s = 0..14).
// Bytes are exact in bf16, every product x_ia c_ib < 2^16 is exact in the fp32
// accumulator, and v_s <= 16 * 8 * 255^2 < 2^23 for at most 16 sources, so every
// partial sum is an exact fp32 integer whatever the summation order. The MMA computes
// all v_s at once as D[p][(t, s)] = sum_(i, a) A[p][(i, a)] B[(i, a)][(t, s)] with
// A[p][(i, a)] = x_ia (the bytes of the sources, K = 8 per source limb) and the
// Toeplitz-shaped constant B[(i, a)][(t, s)] = c_i[t]_(s-a) (zero outside 0..7). One
// more K row adds 2^23 to every accumulator (A = 1, B = 2^23): the fp32 bits of
// 2^23 + v_s are then 0x4B000000 + v_s, and v_s needs no float-to-integer conversion.
//
// Layout (no swizzle, K-major core matrices of 8 rows x 16 bytes):
//  A  [k < ap][p < TP][8 bf16]     the bytes of source limb k at point p (16 bytes): K
//     direction stride TP*16 bytes (LBO), M direction 128 bytes (SBO). Written by the
//     inverse column pass (store_pieces), copied per tile with one bulk copy per limb.
//  B  [u < 2][g < 2][k < ap][r < 8][8 bf16] per target pair: target u, output slots
//     s = 8g + r, limb k; K stride 128 bytes (LBO), N stride ap*128 bytes (SBO). A
//     constant table per (digit, target) / target, built with the context.
//  D  TMEM lane p (of a 128-point M block), column (u, s): one accumulator of
//     (TP / 128) x 32 columns per consumer group, so the MMAs of one group's next pair
//     run while the other group recombines and transforms its own.
//
// One CTA per SM walks a contiguous range of (column tile, target pair) items; the
// bytes of a tile's sources stay in shared memory while the CTA converts them onto
// successive pairs of targets. Roles: one issuer thread (its own warp) copies the
// tile's source bytes and issues the MMAs (completion on mbarriers through
// tcgen05.commit); a loader warp decodes each item's targets (a lane per target) and
// copies their constants an item ahead, off the issuer's path; two consumer groups
// take the items in turn: each reads its lanes' 16 sums per target from TMEM,
// recombines them into the exact 128-bit S, applies REDC and writes the tiles, then its
// two halves run the column NTT of the pair's two targets side by side and store them.
// Full / empty mbarriers and a read counter hand the buffers over between the roles.
#include <algorithm>

#include "ks_internal.h"
#include "ks_kern.cuh"

namespace ks {
namespace kern {

// --- tcgen05 -------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, int cols) {  // one warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int cols) {  // one warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory accesses before this fence are ordered before later
// async-proxy ones (MMA operand reads, bulk copies).
__device__ __forceinline__ void proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ u64 smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (u64)((addr >> 4) & 0x3FFF) | ((u64)((lbo >> 4) & 0x3FFF) << 16) |
         ((u64)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, u64 adesc, u64 bdesc, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive on bar once every MMA this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(u64 *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 16 consecutive 32-bit columns of the warp's lane (TMEM lane = warp quadrant * 32 +
// lane); complete after tmem_wait_ld.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The exact S = sum_s v_s 2^(8s) from the fp32 bits r[s] = 0x4B000000 + v_s
// (v_s < 2^23): pairs P_k = v_2k + v_2k+1 2^8 (< 2^32, weight 2^16k; the 0x4B
// exponent byte of the shifted word falls off the top), quads Q_m = P_2m + P_2m+1 2^16
// (weight 2^32m), then S = Q_0 + Q_1 2^32 + Q_2 2^64 + Q_3 2^96. S < 2^128 keeps
// Q_3 2^32 inside the high word.
__device__ __forceinline__ U128 tc_sum(const uint32_t (&r)[16]) {
  constexpr uint32_t E = 0x4B000000u;
  uint32_t P[8];
#pragma unroll
  for (int k = 0; k < 7; ++k) P[k] = r[2 * k] + (r[2 * k + 1] << 8) - E;
  P[7] = r[14] - E;
  u64 Q[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) Q[m] = (u64)P[2 * m] + ((u64)P[2 * m + 1] << 16);
  U128 s;
  s.lo = Q[0] + (Q[1] << 32);
  s.hi = (Q[1] >> 32) + Q[2] + (Q[3] << 32) + (s.lo < Q[0] ? 1ull : 0ull);
  return s;
}

// A progress counter in shared memory, written by one thread and polled by another:
// rd_set publishes v after the writer's earlier shared-memory accesses; rd_wait polls
// until the counter reaches want (at most ~1 s of %globaltimer and 2^24 polls; false if
// it gave up) and orders the caller's later accesses after it.
__device__ __forceinline__ void rd_set(volatile int *c, int v) {
  __threadfence_block();
  *c = v;
}
__device__ __forceinline__ bool rd_wait(volatile int *c, int want) {
  bool ok = *c >= want;
  if (!ok) {
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < (1 << 24) && !ok; ++it) {
      __nanosleep(32);
      ok = *c >= want;
      if (global_ns() - t0 > 1000000000ull) break;
    }
  }
  __threadfence_block();
  return ok;
}

// Column tiles of TP = 2^kTcTpLog points (N1 rows x GC columns; the inverse column
// passes write the source bytes in blocks of this size), kTcTargets = 2 targets per
// work item (ks_internal.h).
// Consumer groups per CTA.
constexpr int kTcGroups = 2;

// Geometry. Consumers: GRP groups of 256 threads taking items round-robin (so that one
// group's waits and barriers overlap the other's arithmetic); a group is two halves of
// 128 threads, one per target of the pair, 8 points per thread (radix-8 NTT rounds).
// Per group: a TMEM accumulator (8 M blocks x 32 columns), a double constant buffer and
// two NTT tiles. The column twiddles are read from the table (L1).
template <int LOGN, int GRP>
struct TcGeo {
  static constexpr int LOGA = geo_loga(LOGN), LOGB = LOGN - LOGA;
  static constexpr int N1 = 1 << LOGA;
  static constexpr int TPLOG = kTcTpLog, TP = 1 << TPLOG;
  static constexpr int LOGGC = TPLOG - LOGA, GC = 1 << LOGGC, PC = GC + 1;
  static constexpr int MB = TP / 128;  // M blocks of 128 points
  static constexpr int PTS = 8, RM = 3;  // points per consumer thread, NTT stages per round
  static constexpr int HT = TP / PTS;    // consumer threads per target
  static constexpr int GT = 2 * HT;      // threads per group
  static constexpr int NT = GRP * GT;    // consumer threads (+ issuer and loader warps)
  static constexpr int TILES = (1 << LOGN) / TP;
  static constexpr int DCOLS = MB * 32;  // TMEM columns per group
  static constexpr int COLS = GRP * DCOLS <= 256 ? 256 : 512;
  static constexpr int TILE_W = N1 * PC;  // words of one target's NTT tile
  static constexpr int APMAX = 10;        // K slots (alpha <= 9)
  __host__ __device__ static constexpr int smem(int ap) {
    return ap * TP * 16 + GRP * 1024 * ap + GRP * 2 * TILE_W * 8;
  }
  static_assert(kTcTargets == 2 && LOGGC >= 1 && MB % 4 == 0 && (HT / 32) % 4 == 0 &&
                    GRP * DCOLS <= 512 && smem(APMAX) <= 227 * 1024 - 256 && NT + 64 <= 1024,
                "tile shape");
};

struct TcItem {
  int tile, set, y0, cnt;
};
__device__ __forceinline__ TcItem tc_item(const TcItems &ti, int it) {
  TcItem r;
  r.tile = it / ti.pairs;
  const int q = it - r.tile * ti.pairs;
  int s = 0;
  while (s + 1 < ti.nsets && ti.set_p0[s + 1] <= q) ++s;
  r.set = s;
  const int k = q - ti.set_p0[s];
  r.y0 = ti.set_y0[s] + kTcTargets * k;
  r.cnt = min(kTcTargets, ti.set_cnt[s] - kTcTargets * k);
  return r;
}

template <int LOGN, int PRO, int GRP>
__global__ void __launch_bounds__(TcGeo<LOGN, GRP>::NT + 64, 1)
    k_bconv_tc(KArgs a, JobSet js, WsOff wo, Tasks tk, TcItems ti) {
  using G = TcGeo<LOGN, GRP>;
  extern __shared__ __align__(16) unsigned char raw[];
  // Per group g, whose k-th item uses constant buffer and info slot b = k mod 2:
  // bar_b[g][b] (the pair's constants landed; releases the pair's info), bar_m[g] (the
  // MMAs into the group's accumulator completed), bar_tm[g] (every warp of the group has
  // read the accumulator and the info of its item). bar_a: a tile's source bytes landed.
  // rd[g]: items of group g whose sums the issuer has seen read (written by the issuer
  // after its bar_tm wait). The loader fetches a group's next constants into the buffer
  // of its item before last once rd shows that item read, so the copy lands while the
  // group finishes its current item. (A counter, not a second wait on bar_tm: the loader
  // may lag the consumers by more than one phase.)
  __shared__ u64 bar_a, bar_b[GRP][2], bar_m[GRP], bar_tm[GRP];
  __shared__ uint32_t tm_slot;
  __shared__ volatile int rd[GRP];
  // per group and slot, written by the loader before it arms bar_b: the pair's decoded
  // work items, how many are real, the tile, whether both moduli take the fast
  // butterflies, and the source set
  __shared__ uint32_t info_w[GRP][2][2];
  __shared__ int info_cnt[GRP][2], info_tile[GRP][2], info_fast[GRP][2], info_set[GRP][2];
  const JobPtr &jp = js.j[blockIdx.z];
  const int AP = a.tc_ap;
  const int it0 = blockIdx.x * ti.per_cta, it1 = min(ti.items, it0 + ti.per_cta);
  unsigned char *sA = raw;
  unsigned char *sB = raw + (size_t)AP * G::TP * 16;  // [GRP][buffer 2][target 2][256 ap]
  u64 *sT = reinterpret_cast<u64 *>(sB + (size_t)GRP * 1024 * AP);  // [GRP][2][TILE_W]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int CW = G::NT / 32;  // consumer warps; warp CW issues, warp CW + 1 loads

  if (warp == 0) tmem_alloc(&tm_slot, G::COLS);
  if (threadIdx.x == 0) {
    for (int g = 0; g < GRP; ++g) rd[g] = 0;
    mbar_init(&bar_a, 1);
    for (int g = 0; g < GRP; ++g) {
      mbar_init(&bar_b[g][0], 1);
      mbar_init(&bar_b[g][1], 1);
      mbar_init(&bar_m[g], 1);
      mbar_init(&bar_tm[g], G::GT / 32);
    }
  }
  // A: zero (finite values in the slots a short digit leaves unused; their B rows are
  // zero), with bf16 1.0 in the first K element of slot alpha (the 2^23 row); B: zero.
  for (int k = threadIdx.x; k < AP * G::TP; k += blockDim.x)
    reinterpret_cast<uint4 *>(sA)[k] = make_uint4(k / G::TP == a.alpha ? 0x3F80u : 0u, 0, 0, 0);
  for (int k = threadIdx.x; k < GRP * 64 * AP; k += blockDim.x)
    reinterpret_cast<uint4 *>(sB)[k] = make_uint4(0, 0, 0, 0);
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tm_slot;
  pdl_wait();

  auto target = [&](const TcItem &x, int u) { return decode(a, tk, x.y0 + min(u, x.cnt - 1)); };
  if (warp == CW + 1) {
    // Loader warp: each item's decoded targets (the info its group and the issuer read)
    // and the pair's constants, into the group's buffer of the item's index mod 2; lane
    // u < 2 decodes and copies target u.
    for (int it = it0; it < it1; ++it) {
      const int g = (it - it0) % GRP, k = (it - it0) / GRP, b = k & 1;
      // buffer b and info slot b were last used by the group's item k - 2: wait until
      // the issuer has seen its sums read (its MMAs, the buffer's readers, are done)
      if (k >= 2) {
        int ok = 1;
        if (lane == 0) ok = rd_wait(&rd[g], k - 1);
        if (!__shfl_sync(0xffffffffu, ok, 0) && lane == 0) atomicExch(a.tab.err, 1);
        __threadfence_block();
      }
      const TcItem x = tc_item(ti, it);
      uint32_t w = 0;
      int f = 1;
      if (lane < 2) {
        w = target(x, lane);
        info_w[g][b][lane] = w;
        f = a.tab.mod[task_limb(w)].m < kFastModulus;
      }
      f = __all_sync(0xffffffffu, f);
      if (lane == 0) {
        info_cnt[g][b] = x.cnt;
        info_tile[g][b] = x.tile;
        info_set[g][b] = x.set;
        info_fast[g][b] = f;
      }
      __threadfence_block();
      __syncwarp();
      if (lane == 0) mbar_expect_tx(&bar_b[g][b], 2u * 256 * AP);  // releases the info
      __syncwarp();
      if (lane < 2) {
        const int t = task_limb(w);
        const u64 *src = PRO == PRO_UP
                             ? a.tab.bup + ((size_t)task_dig(w) * a.qp + t) * 32 * AP
                             : a.tab.bdown + (size_t)t * 32 * AP;
        bulk_g2s(sB + (size_t)((g * 2 + b) * 2 + lane) * 256 * AP, src, 256 * AP, &bar_b[g][b]);
      }
    }
  } else if (warp == CW) {
    // Issuer (one thread): source bytes and MMAs.
    if (lane == 0) {
      const u64 *pbase = jp.ws + (PRO == PRO_UP ? wo.pv : wo.ppv);
      const u64 ad0 = smem_desc(smem_u32(sA), G::TP * 16, 128);
      unsigned pha = 0;
      int cur_tile = -1, cur_set = -1;
      for (int it = it0; it < it1; ++it) {
        const int g = (it - it0) % GRP;
        const unsigned k = (unsigned)(it - it0) / GRP;  // the group's k-th item
        const int b = k & 1;
        // the group has read the sums and the info of its previous item: its accumulator
        // is free, and the loader may refill that item's constant buffer and info slot
        if (k > 0) {
          if (!mbar_wait(&bar_tm[g], (k - 1) & 1)) atomicExch(a.tab.err, 1);
          rd_set(&rd[g], (int)k);
        }
        // the item's constants and info (its tile and source set)
        if (!mbar_wait(&bar_b[g][b], (k >> 1) & 1)) atomicExch(a.tab.err, 1);
        const int xtile = info_tile[g][b], xset = info_set[g][b];
        if (xtile != cur_tile || xset != cur_set) {
          // a new tile's source bytes, once the MMAs of the previous item no longer read A
          if (it > it0) {
            const int gp = (it - 1 - it0) % GRP;
            if (!mbar_wait(&bar_m[gp], ((unsigned)(it - 1 - it0) / GRP) & 1))
              atomicExch(a.tab.err, 1);
          }
          const int j = ti.set_id[xset];
          const int ns = PRO == PRO_UP ? min(a.nq, (j + 1) * a.alpha) - j * a.alpha : a.np;
          const size_t l0 = (size_t)j * (PRO == PRO_UP ? a.alpha : a.np);
          mbar_expect_tx(&bar_a, (unsigned)ns * G::TP * 16);
          for (int s = 0; s < ns; ++s)
            bulk_g2s(sA + (size_t)s * G::TP * 16,
                     pbase + (((l0 + s) * G::TILES + xtile) << G::TPLOG) * 2, G::TP * 16,
                     &bar_a);
          if (!mbar_wait(&bar_a, pha)) atomicExch(a.tab.err, 1);
          pha ^= 1;
          cur_tile = xtile;
          cur_set = xset;
        }
        tc_fence_after();
        const u64 bd0 = smem_desc(smem_u32(sB + (size_t)(g * 2 + b) * 512 * AP), 128, AP * 128);
        const uint32_t d0 = tmem + g * G::DCOLS;
        // descriptors advance by (byte offset >> 4) in their start-address field; the
        // K steps outside, so consecutive MMAs accumulate into different M blocks
        for (int s = 0; s < AP / 2; ++s)
#pragma unroll
          for (int mb = 0; mb < G::MB; ++mb)
            tc_mma(d0 + mb * 32, ad0 + (u64)(2 * s * G::TP + mb * 128), bd0 + (u64)(16 * s),
                   tc_idesc(32), s > 0);
        tc_commit(&bar_m[g]);
      }
    }
  } else {
    // Consumers: recombine the sums of each item, then the two targets' column NTTs.
    const int group = threadIdx.x / G::GT, bar_id = 1 + group;
    const int half = (threadIdx.x % G::GT) / G::HT;  // the target of the pair
    const int q = warp & 3;  // TMEM lane quadrant of the warp (its 32 points of each M block)
    u64 *dst = jp.ws + (PRO == PRO_UP ? wo.tmp : wo.tmp2);
    u64 *tile = sT + (group * 2 + half) * G::TILE_W;
    for (int it = it0 + group, k = 0; it < it1; it += GRP, ++k) {
      // the pair's decoded items (the loader's info, released with its constants)
      const int b = k & 1;
      if (!mbar_wait(&bar_b[group][b], (k >> 1) & 1)) atomicExch(a.tab.err, 1);
      const uint32_t w = info_w[group][b][half];
      const int cnt = info_cnt[group][b], xtile = info_tile[group][b];
      const bool fast = info_fast[group][b] != 0;
      const ModInfo mi = a.tab.mod[task_limb(w)];
      if (!mbar_wait(&bar_m[group], k & 1)) atomicExch(a.tab.err, 1);
      tc_fence_after();
#pragma unroll
      for (int b0 = 0; b0 < G::MB; b0 += 4) {
        uint32_t v[4][16];
#pragma unroll
        for (int bb = 0; bb < 4; ++bb)
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + group * G::DCOLS + (b0 + bb) * 32 +
                        half * 16,
                    v[bb]);
        tmem_wait_ld();
        if (b0 + 4 == G::MB) {  // the warp's last reads of the accumulator
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_tm[group]);
        }
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const u64 z = redc(tc_sum(v[bb]), mi.m, mi.minv);
          const int p = (b0 + bb) * 128 + 32 * q + lane;
          tile[(p >> G::LOGGC) * G::PC + (p & (G::GC - 1))] = z;
        }
      }
      round_sync<G::GT>(bar_id);
      // both halves take the same butterflies (their rounds share the barrier): the fast
      // ones only when both moduli allow them; twiddles from the column table
      const ulonglong2 *tw = a.tab.twc_f + ((size_t)task_limb(w) << G::LOGA);
      if (fast)
        tile_fwd_t<G::LOGA, G::LOGGC, G::PC, G::HT, false, G::RM, true, 0, true, G::GT>(
            tile, tw, mi.m, bar_id);
      else
        tile_fwd_t<G::LOGA, G::LOGGC, G::PC, G::HT, false, G::RM, false, 0, true, G::GT>(
            tile, tw, mi.m, bar_id);
      if (half < cnt) {
        u64 *d = dst + (size_t)task_slot(w) * a.N;
        const int c0 = xtile * G::GC, lt = threadIdx.x & (G::HT - 1);
#pragma unroll
        for (int r = 0; r < G::TP / 2 / G::HT; ++r) {
          const int e = 2 * (lt + r * G::HT), y = e >> G::LOGGC, c = e & (G::GC - 1);
          ulonglong2 val;
          val.x = tile[y * G::PC + c];
          val.y = tile[y * G::PC + c + 1];
          *reinterpret_cast<ulonglong2 *>(d + ((size_t)y << G::LOGB) + c0 + c) = val;
        }
      }
      round_sync<G::GT>(bar_id);  // the group's tiles are free for its next item
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, G::COLS);
  pdl_trigger();
}

template <int LOGN>
cudaError_t prepare_one() {
  using G = TcGeo<LOGN, kTcGroups>;
  cudaError_t e;
  if ((e = smem_attr(k_bconv_tc<LOGN, PRO_UP, kTcGroups>, G::smem(G::APMAX)))) return e;
  return smem_attr(k_bconv_tc<LOGN, PRO_DOWN, kTcGroups>, G::smem(G::APMAX));
}

template <int LOGN>
cudaError_t launch_one(const ks_context *c, const JobSet &js, const WsOff &wo, const Tasks &tk,
                       const TcItems &ti, int grid, bool up, cudaStream_t s) {
  constexpr int GRP = kTcGroups;
  using G = TcGeo<LOGN, GRP>;
  const int smem = G::smem(c->tc_ap);
  if (up)
    return launch_pdl(k_bconv_tc<LOGN, PRO_UP, GRP>, dim3(grid, 1, js.n), dim3(G::NT + 64), smem,
                      s, args_of(c), js, wo, tk, ti);
  return launch_pdl(k_bconv_tc<LOGN, PRO_DOWN, GRP>, dim3(grid, 1, js.n), dim3(G::NT + 64), smem,
                    s, args_of(c), js, wo, tk, ti);
}

}  // namespace kern

namespace {
// The source sets of a launch and their work items (the Tasks decode order).
bool build_items(const ks_context *c, const Tasks &tk, bool up, TcItems &ti) {
  ti = TcItems{};
  int y = 0;
  if (up) {
    if (tk.j1 - tk.j0 > kTcMaxSets) return false;
    for (int j = tk.j0; j < tk.j1; ++j) {
      Tasks one = tk;
      one.j0 = j;
      one.j1 = j + 1;
      const int k = ti.nsets++;
      ti.set_id[k] = j;
      ti.set_y0[k] = y;
      ti.set_cnt[k] = kern::count_tasks(c, one);
      y += ti.set_cnt[k];
    }
  } else {
    const int n = tk.i1 - tk.i0;
    for (int cc = 0; cc < 2; ++cc) {
      ti.set_id[cc] = cc;
      ti.set_y0[cc] = cc * n;
      ti.set_cnt[cc] = n;
    }
    ti.nsets = 2;
  }
  ti.set_p0[0] = 0;
  for (int k = 0; k < ti.nsets; ++k)
    ti.set_p0[k + 1] = ti.set_p0[k] + (ti.set_cnt[k] + kTcTargets - 1) / kTcTargets;
  ti.pairs = ti.set_p0[ti.nsets];
  ti.tiles = c->N >> c->tc_tplog;
  ti.items = ti.tiles * ti.pairs;
  return true;
}

int sm_count(int dev) {
  static int cached[64] = {};
  if (dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 148;
  }
  return cached[dev];
}
}  // namespace

cudaError_t launch_bconv_tc(const ks_context *c, const JobSet &js, const WsOff &wo,
                            const Tasks &tk, bool up, cudaStream_t s) {
  TcItems ti;
  if (js.n == 0 || c->tc_ap == 0 || !build_items(c, tk, up, ti)) return cudaErrorInvalidValue;
  if (ti.items == 0) return cudaSuccess;
  // one CTA per SM for each job's share of the SMs
  const int per_job = std::max(1, sm_count(c->device) / js.n);
  ti.per_cta = (ti.items + per_job - 1) / per_job;
  const int grid = (ti.items + ti.per_cta - 1) / ti.per_cta;
#define KS_TC_CASE(LN) \
  case LN:              \
    return kern::launch_one<LN>(c, js, wo, tk, ti, grid, up, s);
  switch (c->logn) {
    KS_TC_CASE(13)
    KS_TC_CASE(14)
    KS_TC_CASE(15)
    KS_TC_CASE(16)
    KS_TC_CASE(17)
    default:
      return cudaErrorInvalidValue;
  }
#undef KS_TC_CASE
}

cudaError_t tc_prepare(int logn) {
  switch (logn) {
    case 13: return kern::prepare_one<13>();
    case 14: return kern::prepare_one<14>();
    case 15: return kern::prepare_one<15>();
    case 16: return kern::prepare_one<16>();
    case 17: return kern::prepare_one<17>();
    default: return cudaSuccess;
  }
}

}  // namespace ks
