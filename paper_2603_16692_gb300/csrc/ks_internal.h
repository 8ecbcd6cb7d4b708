// Internal declarations shared by the KeySwitch library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/ks.h"

typedef unsigned long long u64;

namespace ks {

constexpr int kMaxTasks = 1536;  // tasks per launch (kernel parameter list)
constexpr int kMaxLimbs = 256;   // QP limit (L+1 <= 128, alpha <= 128)

// Per-modulus constants (device).
struct ModInfo {
  u64 m;     // modulus
  u64 minv;  // -m^-1 mod 2^64
  u64 r1;    // 2^64 mod m
  u64 r1s;   // Shoup companion of r1
  u64 r2;    // 2^128 mod m
};

// Work items of one launch. Each entry packs: bits 0-7 target limb, bits 8-15
// digit (ModUp) or polynomial index c (ModDown), bits 16-31 buffer slot.
struct TaskList {
  int n;
  uint32_t t[kMaxTasks];
};

__host__ __device__ inline uint32_t pack_task(int limb, int dig, int slot) {
  return (uint32_t)limb | ((uint32_t)dig << 8) | ((uint32_t)slot << 16);
}
__host__ __device__ inline int task_limb(uint32_t w) { return (int)(w & 0xff); }
__host__ __device__ inline int task_dig(uint32_t w) { return (int)((w >> 8) & 0xff); }
__host__ __device__ inline int task_slot(uint32_t w) { return (int)(w >> 16); }

// Device-resident constant tables of one context (all pointers into one
// allocation).
struct Tables {
  ModInfo *mod;          // [QP]
  ulonglong2 *twc_f;     // [QP][N1]  column-pass forward twiddles (w, w')
  ulonglong2 *twc_i;     // [QP][N1]  column-pass inverse twiddles
  ulonglong2 *twr_f;     // [QP][N1/GR][N2-1][GR] row-pass forward twiddles by row tile
  ulonglong2 *twr_i;     // [QP][N1/GR][N2-1][GR]
  ulonglong2 *iscale_q;  // [nq]  N^-1 * Qhat_{j,i}^-1 mod q_i   (Shoup pair)
  ulonglong2 *iscale_p;  // [np]  N^-1 * Phat_k^-1 mod p_k
  u64 *cup;              // [beta][QP][alpha] (Qhat_{j,i} mod m_t) 2^128 mod m_t
  u64 *cdown;            // [nq][alpha]       (Phat_k mod q_i) 2^64 mod q_i
  ulonglong2 *pinv;      // [nq] P^-1 mod q_i (Shoup pair)
  ulonglong2 *pmod;      // [nq] P mod q_i (Shoup pair), keygen only
  int *err;              // sticky device error word
};

struct LaunchTable;

}  // namespace ks

struct ks_context {
  int dnum, logn, L, alpha, beta, nq, np, qp;
  int N;
  int loga, logb, loggr;  // two-pass split N = 2^loga * 2^logb; rows per row tile 2^loggr
  const ks::LaunchTable *lt = nullptr;
  int run_up = 1, run_down = 1;  // max terms per exact 128-bit BConv sum
  std::vector<u64> mods;  // host copy, Q then P
  void *table_mem = nullptr;
  size_t table_bytes = 0;
  ks::Tables tab;
  int device = 0;
  // internal workspace (ks_switch with no caller workspace)
  std::mutex ws_mu;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // staging buffers for ks_switch_host
  void *stage = nullptr;
  size_t stage_bytes = 0;
};

namespace ks {

// Host-side helpers (ks_host.cu)
int build_tables(ks_context *ctx);
bool is_prime_u64(u64 n);

struct SlotMap {
  int sj, st, base;  // slot = j*sj + t*st + base
};

// Per-N launchers of the templated NTT kernels (ks_kern.cuh, ks_inst_*.cu).
struct LaunchTable {
  // iNTT of `outer` x `inner` limbs: src + (o*src_outer + i)*N -> dst + (o*dst_outer + i)*N,
  // limb i modulo prime prime_base + i, scaled by scale[i] (Shoup pair). Row pass
  // first (src -> dst), then the column pass in place on dst (none when N <= 4096).
  cudaError_t (*intt_row)(const ks_context *, const u64 *src, int src_outer, u64 *dst,
                          int dst_outer, int outer, int inner, int prime_base,
                          const ulonglong2 *scale, cudaStream_t);
  cudaError_t (*intt_col)(const ks_context *, u64 *dst, int dst_outer, int outer, int inner,
                          int prime_base, const ulonglong2 *scale, cudaStream_t);
  // ModUp column pass: tasks (t, j, slot): BConv of digit j onto limb t + first NTT pass.
  cudaError_t (*modup_col)(const ks_context *, const TaskList &, const u64 *v, u64 *tmp,
                           cudaStream_t);
  // ModUp row pass + key multiply: tasks (t): digits j0..j1-1 into acc.
  cudaError_t (*modup_row)(const ks_context *, const TaskList &, int j0, int j1, SlotMap,
                           bool first, const u64 *d, const u64 *v, const u64 *tmp,
                           const u64 *evk, u64 *acc, cudaStream_t);
  // ModDown column pass: tasks (i, c, slot): BConv of the P-limbs of c onto q_i + NTT pass.
  cudaError_t (*moddown_col)(const ks_context *, const TaskList &, const u64 *vp, u64 *tmp2,
                             cudaStream_t);
  // ModDown row pass + scaling: tasks (i, -, slot of c=0); c = 1 uses slot + span.
  cudaError_t (*moddown_row)(const ks_context *, const TaskList &, int span, const u64 *vp,
                             const u64 *tmp2, const u64 *acc, u64 *out, cudaStream_t);
  // Plain forward NTT in place of buf[slot] for tasks (t, -, slot): column pass (none
  // when N <= 4096), then row pass with canonical output.
  cudaError_t (*ntt_col)(const ks_context *, const TaskList &, u64 *buf, cudaStream_t);
  cudaError_t (*ntt_row)(const ks_context *, const TaskList &, u64 *buf, cudaStream_t);
};
const LaunchTable *launch_table(int logn);

// Element-wise kernels (ks_elem.cu): the unfused building blocks and keygen.
cudaError_t launch_bconv_up(const ks_context *c, const TaskList &tl, const u64 *v, u64 *tmp,
                            cudaStream_t s);
cudaError_t launch_bconv_down(const ks_context *c, const TaskList &tl, const u64 *vp,
                              u64 *tmp2, cudaStream_t s);
cudaError_t launch_keymult(const ks_context *c, const TaskList &targets, int j0, int j1,
                           SlotMap sm, bool first, const u64 *d, const u64 *tmp,
                           const u64 *evk, u64 *acc, cudaStream_t s);
cudaError_t launch_moddown_scale(const ks_context *c, const TaskList &tl, const u64 *tmp2,
                                 const u64 *acc, u64 *out, cudaStream_t s);
cudaError_t launch_keygen_lift(const ks_context *c, const int8_t *sf, const int8_t *st,
                               const int32_t *e, u64 *polys, cudaStream_t s);
cudaError_t launch_keygen_combine(const ks_context *c, const u64 *polys, const u64 *a,
                                  u64 *evk, cudaStream_t s);

}  // namespace ks
