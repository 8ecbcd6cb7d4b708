// Internal declarations shared by the KeySwitch library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/ks.h"

typedef unsigned long long u64;

namespace ks {

constexpr int kMaxLimbs = 256;   // QP limit (L+1 <= 128, alpha <= 128)

// Per-modulus constants (device).
struct ModInfo {
  u64 m;     // modulus
  u64 minv;  // -m^-1 mod 2^64
  u64 r1;    // 2^64 mod m
  u64 r1s;   // Shoup companion of r1
  u64 r2;    // 2^128 mod m
  u64 mu;    // floor(2^64 / m)
};

// Moduli below this take the fast butterflies (no per-stage reduction, approximate
// Shoup quotients); the bounds they rely on are stated in ks_ntt.cuh.
constexpr u64 kFastModulus = (u64)1 << 51;

// Work items of one launch, decoded from blockIdx.y (see ks_kern.cuh, decode()).
// A decoded item packs: bits 0-7 limb, bits 8-15 digit (ModUp) or polynomial
// index c (ModDown), bits 16-31 buffer slot.
__host__ __device__ inline uint32_t pack_task(int limb, int dig, int slot) {
  return (uint32_t)limb | ((uint32_t)dig << 8) | ((uint32_t)slot << 16);
}
__host__ __device__ inline int task_limb(uint32_t w) { return (int)(w & 0xff); }
__host__ __device__ inline int task_dig(uint32_t w) { return (int)((w >> 8) & 0xff); }
__host__ __device__ inline int task_slot(uint32_t w) { return (int)(w >> 16); }

struct SlotMap {
  int sj, st, base;  // slot = j*sj + t*st + base
};

// Task descriptors. TASK_UP: pairs (digit j, target t) with j in [j0, j1),
// t in [t0, t1) minus digit j's own limbs, slot by `sm`. TASK_TARGET: targets
// t in [t0, t1). TASK_DOWN: pairs (c, i), c in {0, 1}, i in [i0, i1), slot
// c*span + i - ibase. TASK_DOWN1: limbs i in [i0, i1) (both c in one CTA).
// TASK_LINEAR: limbs y in [0, n), prime y % qp, slot y.
enum { TASK_UP = 0, TASK_TARGET = 1, TASK_DOWN = 2, TASK_DOWN1 = 3, TASK_LINEAR = 4 };
struct Tasks {
  int mode;
  int t0, t1, j0, j1;
  SlotMap sm;
  int first;  // key multiply: 1 = write acc, 0 = add into acc
  int i0, i1, span, ibase;
  int n;      // TASK_LINEAR count
};

// Per-job device pointers; the job is blockIdx.z.
constexpr int kMaxBatch = 16;
struct JobPtr {
  const u64 *d;    // [L+1][N] input
  const u64 *evk;  // [beta][2][EQP][N] (EQP = QP, or the top level's QP for a level view)
  u64 *out;        // [2][L+1][N]
  u64 *ws;         // this job's workspace
  const u64 *add;  // optional addend [2][L+1][N] (may alias out): out_c += add_c when
  int addmask;     // bit c of addmask is set (HMUL / HROT epilogues); 0 = plain store
  const u64 *dsrc; // optional: the input in (pinned, device-mapped) host memory; the
                   // input iNTT reads it and leaves a device copy in d
};
struct JobSet {
  int n;
  JobPtr j[kMaxBatch];
};
// Word offsets of the workspace pieces.
struct WsOff {
  long long v, tmp, acc, vp, tmp2;
  // tensor-core basis conversions: the bf16 bytes of v and of vp (see ks_tc.cu)
  long long pv, ppv;
};
// Which workspace piece a plain NTT pass works on.
enum { BUF_TMP = 0, BUF_TMP2 = 1 };

struct Tables {
  ModInfo *mod;          // [QP]
  ulonglong2 *twc_f;     // [QP][N1]  column-pass forward twiddles (w, w')
  ulonglong2 *twc_i;     // [QP][N1]  column-pass inverse twiddles
  ulonglong2 *twr_f;     // [QP][N1/GR][N2-1][GR] row-pass twiddles by row tile (the
                         // inverse row pass reads them mirrored)
  ulonglong2 *iscale_q;  // [nq]  N^-1 * Qhat_{j,i}^-1 mod q_i   (Shoup pair)
  ulonglong2 *iscale_p;  // [np]  N^-1 * Phat_k^-1 mod p_k
  u64 *cup;              // [beta][QP][alpha] (Qhat_{j,i} mod m_t) 2^128 mod m_t
  u64 *cdown;            // [nq][alpha]       (Phat_k mod q_i) 2^64 mod q_i
  ulonglong2 *pinv;      // [nq] P^-1 mod q_i (Shoup pair)
  ulonglong2 *pmod;      // [nq] P mod q_i (Shoup pair), keygen only
  // Tensor-core basis conversions (ks_tc.cu): the constants of cup / cdown as bf16
  // bytes in the MMA's B layout, 32 * tc_ap words per (digit, target) / target.
  u64 *bup;              // [beta][QP][32 tc_ap] (empty when the context has no TC path)
  u64 *bdown;            // [nq][32 tc_ap]
  int *err;              // sticky device error word
};

// Tensor-core basis conversion: at most this many source sets (digits) per context.
constexpr int kTcMaxSets = 64;
// Tensor-core BConv work items: column tiles of 2^kTcTpLog points, kTcTargets targets
// (of one source set) per item.
constexpr int kTcTpLog = 10;
constexpr int kTcTargets = 2;
// Work of one tensor-core BConv launch: the target groups of every source set, over all
// column tiles; item = (tile, target group), tile-major (see ks_tc.cu).
struct TcItems {
  int nsets, pairs, tiles, items, per_cta;  // pairs: target groups per tile
  int set_id[kTcMaxSets];       // digit j (ModUp) or polynomial c (ModDown)
  int set_y0[kTcMaxSets];       // first work item (Tasks index) of the set
  int set_cnt[kTcMaxSets];      // work items of the set
  int set_p0[kTcMaxSets + 1];   // target groups before the set
};

struct LaunchTable;

}  // namespace ks

struct ks_context {
  int dnum, logn, L, alpha, beta, nq, np, qp;
  // Key layout: evk[j][c][t'] with t' = t for Q-limbs, eqp_base + (t - nq) for P-limbs,
  // limb stride eqp. A top-level context has eqp = qp, epb = nq; a level view (KeySwitch
  // at level l < L with the top level's keys) keeps the top level's layout.
  int eqp = 0, epb = 0;
  int top_L = -1;  // level of the context whose keys this one uses (-1: itself)
  int N;
  int loga, logb, loggr;  // two-pass split N = 2^loga * 2^logb; rows per row tile 2^loggr
  // Launchers by register-round radix (index log2 radix - 2: radix 4 has twice the
  // threads per tile of radix 8, radix 16 half) and column tile (0: default, 1: the
  // alternative); lt = radix 8, default tiles.
  const ks::LaunchTable *ltab[3][2] = {};
  const ks::LaunchTable *lt = nullptr;
  int run_up = 1, run_down = 1;  // max terms per exact 128-bit BConv sum
  // Tensor-core basis conversions: K slots per source set (alpha + 1 rounded up to
  // even; 0 = not available for this context) and log2 of the points per column tile.
  int tc_ap = 0, tc_tplog = 0;
  std::vector<u64> mods;  // host copy, Q then P
  void *table_mem = nullptr;
  size_t table_bytes = 0;
  ks::Tables tab;
  int device = 0;
  // internal workspace (ks_switch with no caller workspace)
  std::mutex ws_mu;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // timing-based choice of the dataflow (ks_tune); 0 = not tuned
  int tuned_variant = 0, tuned_chunks = 0, tuned_batch = 0;
  // the installed selector network's choice (ks_select); sel_gen = the selector it
  // came from (0 = none)
  int sel_variant = 0, sel_chunks = 0;
  unsigned sel_gen = 0;
  float tuned_ms = 0;
  // staging buffers for ks_switch_host
  void *stage = nullptr;
  size_t stage_bytes = 0;
  // CUDA graphs of repeated single-operation calls (ks_switch / ks_hmul / ks_hrot
  // with the same plan, buffers and stream), captured on the second such call
  std::mutex gmu;
  struct CachedGraph {
    cudaGraphExec_t exec = nullptr;  // null: seen once, not captured yet
    unsigned long long last = 0;
    bool direct = false;  // capture failed (e.g. pageable host memory): launch directly
  };
  std::map<std::array<uintptr_t, 10>, CachedGraph> gcache;
  unsigned long long gclock = 0;
  cudaStream_t gstream = nullptr;  // capture stream
  // second stream of plans with KS_SPLIT_DOWN (the Q-limb key multiply runs there while
  // the P-limb ModDown chain runs on the caller's stream), its fork / join events, and
  // the lock that keeps one call's record / wait pairs together
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::mutex side_mu;
};

namespace ks {

// Launch `kernel` on s with programmatic stream serialization allowed: it may start
// while the previous kernel of the stream finishes (the kernels synchronise with
// griddepcontrol.wait before touching shared buffers).
template <class... KT, class... AT>
inline cudaError_t launch_pdl(void (*kernel)(KT...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, AT &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<AT &&>(args)...);
}

// Host-side helpers (ks_host.cu)
int build_tables(ks_context *ctx);
bool is_prime_u64(u64 n);

// Per-N launchers of the templated NTT kernels (ks_kern.cuh, ks_inst_*.cu). Every
// launch covers the jobs of `js` (grid z) and the work items of `tk` (grid y).
struct LaunchTable {
  // Opt in to the dynamic shared memory of every kernel of this N (once).
  cudaError_t (*prepare)();
  // Number of work items a descriptor decodes to (grid y).
  int (*count)(const ks_context *, const Tasks &);
  // iNTT of the L+1 input limbs (which = 0: d -> v, scaled by N^-1 Qhat^-1) or of the
  // alpha P-limbs of both accumulators (which = 1: acc -> vp, scaled by N^-1 Phat^-1).
  // Row pass (src -> dst), then the column pass in place (none when N <= 4096).
  cudaError_t (*intt_row)(const ks_context *, const JobSet &, const WsOff &, int which,
                          cudaStream_t);
  cudaError_t (*intt_col)(const ks_context *, const JobSet &, const WsOff &, int which,
                          cudaStream_t);
  // The same column pass writing the bf16 bytes of its output (pv / ppv) for the
  // tensor-core basis conversion instead of v / vp.
  cudaError_t (*intt_col_tc)(const ks_context *, const JobSet &, const WsOff &, int which,
                             cudaStream_t);
  // ModUp column pass (TASK_UP): BConv of digit j onto limb t + first NTT pass -> tmp.
  cudaError_t (*modup_col)(const ks_context *, const JobSet &, const WsOff &, const Tasks &,
                           cudaStream_t);
  // ModUp row pass + key multiply (TASK_TARGET): digits j0..j1-1 into acc.
  cudaError_t (*modup_row)(const ks_context *, const JobSet &, const WsOff &, const Tasks &,
                           cudaStream_t);
  // ModDown column pass (TASK_DOWN): BConv of the P-limbs of c onto q_i + NTT pass -> tmp2.
  cudaError_t (*moddown_col)(const ks_context *, const JobSet &, const WsOff &, const Tasks &,
                             cudaStream_t);
  // ModDown row pass + scaling (TASK_DOWN1): out = (acc - NTT(.)) * P^-1.
  cudaError_t (*moddown_row)(const ks_context *, const JobSet &, const WsOff &, const Tasks &,
                             cudaStream_t);
  // Plain forward NTT, in place on workspace piece `buf` (BUF_TMP / BUF_TMP2) for the
  // items of `tk` (TASK_UP, TASK_DOWN or TASK_LINEAR): column pass, then row pass with
  // canonical output.
  cudaError_t (*ntt_col)(const ks_context *, const JobSet &, const WsOff &, const Tasks &,
                         int buf, cudaStream_t);
  cudaError_t (*ntt_row)(const ks_context *, const JobSet &, const WsOff &, const Tasks &,
                         int buf, cudaStream_t);
};
// ks_switch on the caller's workspace `ws` (ws_bytes >= ks_workspace_size) that only
// launches kernels, all on `stream` (a KS_SPLIT_DOWN plan runs unsplit): no graph
// cache, no arena (ks_api.cu).
int switch_launch_only(ks_context *c, const uint64_t *d, const uint64_t *evk, uint64_t *out,
                       int variant, int chunks, void *ws, size_t ws_bytes, void *stream);
// True when ctx's selected plan came from the selector installed now (ks_select.cu).
bool selected_current(const ks_context *c);

// rl = log2 of the radix of the register rounds (3: 8 points per thread, 2: 4 points
// per thread, twice the threads per tile; 4: 16 points); ca = 1: the alternative
// column tile (geo_tile_log_col_alt).
const LaunchTable *launch_table(int logn, int rl, int ca);

// Tensor-core basis conversion + first forward NTT pass (ks_tc.cu), in place of the
// fused column passes modup_col (up = true, TASK_UP -> tmp) and moddown_col (TASK_DOWN ->
// tmp2); reads the bytes the intt_col_tc pass wrote. Needs ctx->tc_ap > 0.
cudaError_t launch_bconv_tc(const ks_context *c, const JobSet &js, const WsOff &o,
                            const Tasks &tk, bool up, cudaStream_t s);
// Opt in to the shared memory of the tensor-core kernels of this N (once per context).
cudaError_t tc_prepare(int logn);

// Element-wise kernels (ks_elem.cu): the unfused building blocks and keygen.
cudaError_t launch_bconv_up(const ks_context *c, const JobSet &js, const WsOff &o,
                            const Tasks &tk, int count, cudaStream_t s);
cudaError_t launch_bconv_down(const ks_context *c, const JobSet &js, const WsOff &o,
                              const Tasks &tk, int count, cudaStream_t s);
cudaError_t launch_keymult(const ks_context *c, const JobSet &js, const WsOff &o,
                           const Tasks &tk, cudaStream_t s);
cudaError_t launch_moddown_scale(const ks_context *c, const JobSet &js, const WsOff &o,
                                 const Tasks &tk, int count, cudaStream_t s);
// Persistent batch (ks_persist.cu).
struct PersistBatch;
bool persist_supported(const ks_context *c);
int persist_radix(int logn);
PersistBatch *persist_new();
void persist_free(PersistBatch *pb);
void persist_build(PersistBatch &pb, const std::vector<const ks_context *> &ctx,
                   const std::vector<JobPtr> &jp, const std::vector<WsOff> &wo);
size_t persist_bytes(const PersistBatch &pb);
size_t persist_state_offset(const PersistBatch &pb);
int persist_counts(const PersistBatch &pb, int *njobs, int *nwork, int *ncnt);
int persist_upload(const PersistBatch &pb, void *dev, cudaStream_t s);
// Stage-major form: the work list's stage boundaries (kPersistStages + 1 offsets, then
// the ends of the key-multiply and ModDown-row items of N >= 2^16 jobs, which come first
// in their stages), and the launch of one persistent kernel per stage (two for those
// stages; no waits inside a kernel).
constexpr int kPersistStages = 8;
void persist_stage_offsets(const PersistBatch &pb, int *off);
int persist_launch_staged(void *dev, int njobs, const int *stage_off, int ncnt,
                          size_t state_offset, cudaStream_t s);
int persist_launch(void *dev, int njobs, int nwork, int ncnt, size_t state_offset,
                   unsigned long long limit_ns, bool stall, cudaStream_t s);
int persist_status(const void *dev, size_t state_offset, cudaStream_t s);

// Key generation: lift s_from (optionally through the automorphism x -> x^k, given
// by kinv = k^-1 mod 2N; kinv 0 = identity), s_to and the errors to residues.
cudaError_t launch_keygen_lift(const ks_context *c, const int8_t *sf, const int8_t *st,
                               const int32_t *e, unsigned kinv, u64 *polys, cudaStream_t s);
// Square the NTT-form s_from residues in place (relinearisation key: s_from = s^2).
cudaError_t launch_keygen_square(const ks_context *c, u64 *polys, cudaStream_t s);
cudaError_t launch_keygen_combine(const ks_context *c, const u64 *polys, const u64 *a,
                                  u64 *evk, cudaStream_t s);
// HMUL tensor product over Q (NTT form): out_0 = x0 y0, out_1 = x0 y1 + x1 y0, d2 = x1 y1.
cudaError_t launch_tensor(const ks_context *c, const u64 *x, const u64 *y, u64 *out, u64 *d2,
                          cudaStream_t s);
// Galois automorphism x -> x^k of both polynomials of ct (NTT form, bit-reversed slots):
// y0 = sigma(ct_0), y1 = sigma(ct_1).
cudaError_t launch_automorph(const ks_context *c, const u64 *ct, unsigned k, u64 *y0, u64 *y1,
                             cudaStream_t s);

}  // namespace ks
