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
//  D  TMEM lane p (of a 128-point M block), column (u, s): two buffers of
//     (TP / 128) x 32 columns, so the MMAs of the next pair run while this pair's sums
//     are recombined.
//
// One CTA per SM walks a contiguous range of (column tile, target pair) items; the
// bytes of a tile's sources stay in shared memory while the CTA converts them onto
// successive pairs of targets. Per item: thread 0 issues the MMAs (one elected thread,
// completion on an mbarrier through tcgen05.commit); every thread reads its lane's 16
// sums per target from TMEM, recombines them into the exact 128-bit S, applies REDC,
// and writes the tile; then the two halves of the block run the column NTT of the two
// targets side by side and store them.
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

// Geometry: column tiles of TP = 2^TPLOG points (N1 rows x GC columns).
template <int LOGN, int TPLOG>
struct TcGeo {
  static constexpr int LOGA = geo_loga(LOGN), LOGB = LOGN - LOGA;
  static constexpr int N1 = 1 << LOGA;
  static constexpr int TP = 1 << TPLOG;
  static constexpr int LOGGC = TPLOG - LOGA, GC = 1 << LOGGC, PC = GC + 1;
  static constexpr int MB = TP / 128;  // M blocks of 128 points
  static constexpr int HT = TP / 4;    // threads per target of a pair (4 points each)
  static constexpr int NT = 2 * HT;
  static constexpr int TILES = (1 << LOGN) / TP;
  static constexpr int COLS = 2 * MB * 32;  // TMEM columns: two buffers
  static constexpr int TILE_W = N1 * PC;    // words of one target's NTT tile
  static constexpr int APMAX = TPLOG >= 10 ? 10 : 16;
  // shared memory for ap K slots per source set
  __host__ __device__ static constexpr int smem(int ap) {
    return ap * TP * 16 + 4 * 256 * ap + 4 * N1 * 16 + 2 * TILE_W * 8;
  }
  static_assert(LOGGC >= 1 && MB % 4 == 0, "tile shape");
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
  r.y0 = ti.set_y0[s] + 2 * k;
  r.cnt = min(2, ti.set_cnt[s] - 2 * k);
  return r;
}

template <int LOGN, int PRO, int TPLOG>
__global__ void __launch_bounds__(TcGeo<LOGN, TPLOG>::NT, 1)
    k_bconv_tc(KArgs a, JobSet js, WsOff wo, Tasks tk, TcItems ti) {
  using G = TcGeo<LOGN, TPLOG>;
  extern __shared__ __align__(1024) unsigned char raw[];
  __shared__ u64 bar_a, bar_b[2], bar_m[2];
  __shared__ uint32_t tm_slot;
  const JobPtr &jp = js.j[blockIdx.z];
  const int AP = a.tc_ap;
  const int it0 = blockIdx.x * ti.per_cta, it1 = min(ti.items, it0 + ti.per_cta);
  unsigned char *sA = raw;
  unsigned char *sB = raw + (size_t)AP * G::TP * 16;
  ulonglong2 *sTW = reinterpret_cast<ulonglong2 *>(sB + 4 * 256 * AP);
  u64 *sT = reinterpret_cast<u64 *>(sTW + 4 * G::N1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = threadIdx.x / G::HT;  // the target of the pair this thread works on

  if (warp == 0) tmem_alloc(&tm_slot, G::COLS);
  if (threadIdx.x == 0) {
    mbar_init(&bar_a, 1);
    mbar_init(&bar_b[0], 1);
    mbar_init(&bar_b[1], 1);
    mbar_init(&bar_m[0], 1);
    mbar_init(&bar_m[1], 1);
  }
  // A: zero (finite values in the slots a short digit leaves unused; their B rows are
  // zero), with bf16 1.0 in the first K element of slot alpha (the 2^23 row); B: zero.
  for (int k = threadIdx.x; k < AP * G::TP; k += G::NT)
    reinterpret_cast<uint4 *>(sA)[k] = make_uint4(k / G::TP == a.alpha ? 0x3F80u : 0u, 0, 0, 0);
  for (int k = threadIdx.x; k < 4 * 16 * AP; k += G::NT)
    reinterpret_cast<uint4 *>(sB)[k] = make_uint4(0, 0, 0, 0);
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tm_slot;
  pdl_wait();

  const u64 *pbase = jp.ws + (PRO == PRO_UP ? wo.pv : wo.ppv);
  u64 *dst = jp.ws + (PRO == PRO_UP ? wo.tmp : wo.tmp2);
  auto nsrc = [&](int set) {
    const int j = ti.set_id[set];
    return PRO == PRO_UP ? min(a.nq, (j + 1) * a.alpha) - j * a.alpha : a.np;
  };
  auto target = [&](const TcItem &x, int u) { return decode(a, tk, x.y0 + min(u, x.cnt - 1)); };
  // thread 0: bulk copies of a tile's source bytes (bar_a) / of a pair's constants and
  // twiddles (bar_b[buf])
  auto load_a = [&](const TcItem &x) {
    const int ns = nsrc(x.set);
    const size_t l0 = (size_t)ti.set_id[x.set] * (PRO == PRO_UP ? a.alpha : a.np);
    mbar_expect_tx(&bar_a, (unsigned)ns * G::TP * 16);
    for (int k = 0; k < ns; ++k)
      bulk_g2s(sA + (size_t)k * G::TP * 16,
               pbase + (((l0 + k) * G::TILES + x.tile) << TPLOG) * 2, G::TP * 16, &bar_a);
  };
  auto load_b = [&](const TcItem &x, int buf) {
    mbar_expect_tx(&bar_b[buf], 2u * (256 * AP + G::N1 * 16));
    for (int u = 0; u < 2; ++u) {
      const uint32_t w = target(x, u);
      const int t = task_limb(w);
      const u64 *b = PRO == PRO_UP ? a.tab.bup + ((size_t)task_dig(w) * a.qp + t) * 32 * AP
                                   : a.tab.bdown + (size_t)t * 32 * AP;
      bulk_g2s(sB + (size_t)(buf * 2 + u) * 256 * AP, b, 256 * AP, &bar_b[buf]);
      bulk_g2s(sTW + (buf * 2 + u) * G::N1, a.tab.twc_f + ((size_t)t << G::LOGA), G::N1 * 16,
               &bar_b[buf]);
    }
  };
  // barrier phases: bit buf of phb / phm is the next phase of bar_b[buf] / bar_m[buf]
  unsigned pha = 0, phb = 0, phm = 0;
  auto issue_mma = [&](int buf, bool wait_a) {
    if (wait_a) {
      if (!mbar_wait(&bar_a, pha)) atomicExch(a.tab.err, 1);
      pha ^= 1;
    }
    if (!mbar_wait(&bar_b[buf], (phb >> buf) & 1)) atomicExch(a.tab.err, 1);
    phb ^= 1u << buf;
    tc_fence_after();
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB + (size_t)buf * 2 * 256 * AP);
    for (int b = 0; b < G::MB; ++b)
      for (int k = 0; k < AP / 2; ++k)
        tc_mma(tmem + buf * (G::MB * 32) + b * 32,
               smem_desc(a0 + 2 * k * G::TP * 16 + b * 2048, G::TP * 16, 128),
               smem_desc(b0 + 2 * k * 128, 128, AP * 128), tc_idesc(32), k > 0);
    tc_commit(&bar_m[buf]);
  };

  if (it0 < it1 && threadIdx.x == 0) {
    const TcItem x = tc_item(ti, it0);
    load_a(x);
    load_b(x, it0 & 1);
    issue_mma(it0 & 1, true);
  }
  const int q = warp & 3, r4 = ((warp % (G::HT / 32)) >> 2) * 4;  // TMEM quadrant, M blocks
  for (int it = it0; it < it1; ++it) {
    const int buf = it & 1;
    const TcItem x = tc_item(ti, it);
    const bool more = it + 1 < it1;
    TcItem nx = x;
    bool nx_unit = false;
    if (more) {
      nx = tc_item(ti, it + 1);
      nx_unit = nx.tile != x.tile || nx.set != x.set;
    }
    if (threadIdx.x == 0 && more) load_b(nx, buf ^ 1);
    if (!mbar_wait(&bar_m[buf], (phm >> buf) & 1)) atomicExch(a.tab.err, 1);
    phm ^= 1u << buf;
    tc_fence_after();
    // the MMAs of item `it` were the last to read A: a new tile's bytes may land now
    if (threadIdx.x == 0 && nx_unit) load_a(nx);
    const uint32_t w = target(x, half);
    const int t = task_limb(w);
    const ModInfo mi = a.tab.mod[t];
    u64 *tile = sT + half * G::TILE_W;
    {
      uint32_t v[4][16];
#pragma unroll
      for (int bb = 0; bb < 4; ++bb)
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + buf * (G::MB * 32) + (r4 + bb) * 32 +
                      half * 16,
                  v[bb]);
      tmem_wait_ld();
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) {
        const u64 z = redc(tc_sum(v[bb]), mi.m, mi.minv);
        const int p = (r4 + bb) * 128 + 32 * q + lane;
        tile[(p >> G::LOGGC) * G::PC + (p & (G::GC - 1))] = z;
      }
    }
    if (threadIdx.x == 0 && more) issue_mma(buf ^ 1, nx_unit);
    tc_fence_before();
    __syncthreads();
    // both halves take the same butterflies (their rounds share the block's barriers):
    // the fast ones only when both moduli allow them
    const ulonglong2 *tw = sTW + (buf * 2 + half) * G::N1;
    if (mi.m < kFastModulus && a.tab.mod[task_limb(target(x, half ^ 1))].m < kFastModulus)
      tile_fwd_t<G::LOGA, G::LOGGC, G::PC, G::HT, false, 2, true, 0, true>(tile, tw, mi.m);
    else
      tile_fwd_t<G::LOGA, G::LOGGC, G::PC, G::HT, false, 2, false, 0, true>(tile, tw, mi.m);
    if (half < x.cnt) {
      u64 *d = dst + (size_t)task_slot(w) * a.N;
      const int c0 = x.tile * G::GC, lt = threadIdx.x & (G::HT - 1);
#pragma unroll
      for (int k = 0; k < G::TP / 2 / G::HT; ++k) {
        const int e = 2 * (lt + k * G::HT), y = e >> G::LOGGC, g = e & (G::GC - 1);
        ulonglong2 val;
        val.x = tile[y * G::PC + g];
        val.y = tile[y * G::PC + g + 1];
        *reinterpret_cast<ulonglong2 *>(d + ((size_t)y << G::LOGB) + c0 + g) = val;
      }
    }
    proxy_fence();
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, G::COLS);
  pdl_trigger();
}

template <int LOGN, int TPLOG>
cudaError_t prepare_one() {
  using G = TcGeo<LOGN, TPLOG>;
  cudaError_t e;
  if ((e = smem_attr(k_bconv_tc<LOGN, PRO_UP, TPLOG>, G::smem(G::APMAX)))) return e;
  return smem_attr(k_bconv_tc<LOGN, PRO_DOWN, TPLOG>, G::smem(G::APMAX));
}

template <int LOGN, int TPLOG>
cudaError_t launch_one(const ks_context *c, const JobSet &js, const WsOff &wo, const Tasks &tk,
                       const TcItems &ti, int grid, bool up, cudaStream_t s) {
  using G = TcGeo<LOGN, TPLOG>;
  const int smem = G::smem(c->tc_ap);
  if (up)
    return launch_pdl(k_bconv_tc<LOGN, PRO_UP, TPLOG>, dim3(grid, 1, js.n), dim3(G::NT), smem, s,
                      args_of(c), js, wo, tk, ti);
  return launch_pdl(k_bconv_tc<LOGN, PRO_DOWN, TPLOG>, dim3(grid, 1, js.n), dim3(G::NT), smem, s,
                    args_of(c), js, wo, tk, ti);
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
  for (int k = 0; k < ti.nsets; ++k) ti.set_p0[k + 1] = ti.set_p0[k] + (ti.set_cnt[k] + 1) / 2;
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
  const bool big = c->tc_tplog >= 10;
#define KS_TC_CASE(LN)                                                     \
  case LN:                                                                \
    return big ? kern::launch_one<LN, 10>(c, js, wo, tk, ti, grid, up, s) \
               : kern::launch_one<LN, 9>(c, js, wo, tk, ti, grid, up, s);
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
  cudaError_t e = cudaSuccess;
  switch (logn) {
    case 13:
      if (!(e = kern::prepare_one<13, 10>())) e = kern::prepare_one<13, 9>();
      break;
    case 14:
      if (!(e = kern::prepare_one<14, 10>())) e = kern::prepare_one<14, 9>();
      break;
    case 15:
      if (!(e = kern::prepare_one<15, 10>())) e = kern::prepare_one<15, 9>();
      break;
    case 16:
      if (!(e = kern::prepare_one<16, 10>())) e = kern::prepare_one<16, 9>();
      break;
    case 17:
      if (!(e = kern::prepare_one<17, 10>())) e = kern::prepare_one<17, 9>();
      break;
    default:
      break;
  }
  return e;
}

}  // namespace ks
