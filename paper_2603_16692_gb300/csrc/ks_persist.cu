// One persistent launch for a batch of KeySwitches of uneven (dnum, N, L): a
// dataflow executor over tile-level work items.
//
// Stages of one job (DPOB, fused, two-pass NTT; N = 2^13..2^17):
//   0 iNTT rows (d)   1 iNTT columns (d)   2 ModUp BConv + NTT columns
//   3 NTT rows + key multiply   4 iNTT rows (P-limbs)   5 iNTT columns (P-limbs)
//   6 ModDown BConv + NTT columns   7 NTT rows + P^-1 scaling
// A work item is one tile of one stage (the same device code as the per-stage
// kernels). It waits on at most two dependency counters and signals one, so an
// item starts as soon as the tiles it reads are written, not when the whole
// previous stage is done:
//   1 (col tile, limb i)      waits for the row tiles of limb i       (stage 0)
//   2 (col tile c, (t, j))    waits for col tile c of digit j's limbs (stage 1)
//   3 (row tile r, target t)  waits for every (col tile, digit) of t  (stage 2)
//   4 (row tile r, P-limb k)  waits for row tile r of target L+1+k    (stage 3)
//   5 (col tile, P-limb k)    waits for the row tiles of P-limb k     (stage 4)
//   6 (col tile c, (c', i))   waits for col tile c of every P-limb    (stage 5)
//   7 (row tile r, limb i)    waits for every col tile of (0, i), (1, i)  (stage 6)
//                             and for row tile r of target i          (stage 3)
// The host builds the items, their counters and the counts they wait for.
//
// Every CTA loops: it claims the next item from a device counter, waits for the
// item's dependencies, runs it and signals. Items are listed stage-major over
// all jobs, so an item only depends on items with smaller indices. Items are
// claimed in index order, and only by CTAs that are running, so the earliest
// unfinished item is held by a running CTA and has nothing left to wait for: the
// loop cannot deadlock, resident grid or not. Each CTA claims its next item while
// it runs the current one; that item too only waits for smaller indices.
// Completion is counted with a release increment after the CTA's barrier, and the
// consumer's acquire load of the counter (then a barrier) orders its reads after
// the producer's writes.
//
// Waits are bounded: a wait that exceeds `limit_ns` of %globaltimer sets the
// device error word and the abort flag, and every CTA then returns; the host
// reads the error with ks_batch_status (KS_ETIMEOUT). Buffers written during the
// launch are read with coherent loads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ks_kern.cuh"

namespace ks {
namespace {

using kern::KArgs;

constexpr int kStages = 8;
constexpr int kPNT = 256;  // threads per CTA of the persistent kernel

// The radix of the rounds for each N and pass: 256 threads per tile at every size
// (tiles of 2^9 points take radix 2, 2^10 radix 4, 2^11 radix 8).
__host__ __device__ constexpr int prl_col(int logn) { return geo_tile_log_col(logn) - 8; }
__host__ __device__ constexpr int prl_row(int logn) { return geo_tile_log_row(logn) - 8; }

struct PJob {
  KArgs a;
  JobPtr jp;
  WsOff wo;
  Tasks up, tg, dn, d1;
  int logn;
};

// One tile of one stage of one job, with its dependencies: counters cnt[w0] and
// cnt[w1] (-1: none) must reach n0 and n1 before it runs; it then adds 1 to
// cnt[sig] (-1: none).
struct PWork {
  uint16_t job, bx, by;
  uint8_t stage, pad;
  int32_t w0, w1, sig;
  uint16_t n0, n1;
};

struct PState {
  int next;
  int abort;
  int err;
  int pad;
  int snext[kStages + 2];  // next item of each stage-major launch
  int cnt[1];          // dependency counters
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Release increment: the CTA's writes (ordered before by the barrier that precedes
// it) are visible to any thread that acquires the counter's new value.
__device__ __forceinline__ void red_release_add(int *p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Polls of one wait before it gives up even if %globaltimer were not advancing.
constexpr long long kMaxPolls = 1ll << 28;

// 1 when *flag >= target, 0 when the wait gave up (time or poll limit, or abort).
__device__ int wait_count(const int *flag, int target, PState *st, unsigned long long limit_ns) {
  if (ld_acquire(flag) >= target) return 1;
  const unsigned long long t0 = globaltimer();
  for (long long it = 0; it < kMaxPolls; ++it) {
    if (ld_acquire(flag) >= target) return 1;
    if (ld_acquire(&st->abort)) return 0;
    if (globaltimer() - t0 > limit_ns) break;
    __nanosleep(200);
  }
  atomicExch(&st->err, 1);
  atomicExch(&st->abort, 1);
  return 0;
}

// One stage body per (N, stage). (Kept inline: separate functions spill less but
// measured slower on GB300, the call boundary costing more than the spills.)
template <int LOGN, int STAGE>
__device__ __forceinline__ void stage_fn(const PJob &J, int which, int bx, int by,
                                      unsigned char *raw, u64 *cst) {
  constexpr int RC = prl_col(LOGN), RR = prl_row(LOGN);
  if constexpr (STAGE == 0) kern::inv_row_body<LOGN, RR, false>(J.a, J.jp, J.wo, which, bx, by, raw);
  if constexpr (STAGE == 1) kern::inv_col_body<LOGN, RC, 0, false>(J.a, J.jp, J.wo, which, bx, by, raw);
  if constexpr (STAGE == 2)
    kern::fwd_col_body<LOGN, RC, kern::PRO_UP, 0, false>(J.a, J.jp, J.wo, J.up, BUF_TMP, bx, by, raw, cst);
  if constexpr (STAGE == 3)
    kern::keymult_body<LOGN, RR, kern::PRO_LOAD, false>(J.a, J.jp, J.wo, J.tg, bx, by, raw, cst);
  if constexpr (STAGE == 6)
    kern::fwd_col_body<LOGN, RC, kern::PRO_DOWN, 0, false>(J.a, J.jp, J.wo, J.dn, BUF_TMP2, bx, by, raw,
                                                cst);
  if constexpr (STAGE == 7)
    kern::moddown_body<LOGN, RR, kern::PRO_LOAD, false>(J.a, J.jp, J.wo, J.d1, bx, by, raw, cst);
}

template <int LOGN>
__device__ __forceinline__ void run_stage(const PJob &J, int stage, int bx, int by,
                                          unsigned char *raw, u64 *cst) {
  switch (stage) {
    case 0: stage_fn<LOGN, 0>(J, 0, bx, by, raw, cst); break;
    case 1: stage_fn<LOGN, 1>(J, 0, bx, by, raw, cst); break;
    case 2: stage_fn<LOGN, 2>(J, 0, bx, by, raw, cst); break;
    case 3: stage_fn<LOGN, 3>(J, 0, bx, by, raw, cst); break;
    case 4: stage_fn<LOGN, 0>(J, 1, bx, by, raw, cst); break;
    case 5: stage_fn<LOGN, 1>(J, 1, bx, by, raw, cst); break;
    case 6: stage_fn<LOGN, 6>(J, 0, bx, by, raw, cst); break;
    default: stage_fn<LOGN, 7>(J, 0, bx, by, raw, cst); break;
  }
}

// Three CTAs per SM (80 registers): measured on GB300 against one (49 ms for the
// 64-job batch) and two (30 ms); three gave 25 ms despite small spills.
__global__ void __launch_bounds__(kPNT, 3) k_persist(const PJob *__restrict__ jobs,
                                                  const PWork *__restrict__ work, int nwork,
                                                  PState *st, unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ u64 cst[kMaxLimbs];
  __shared__ PJob J;
  __shared__ int item, nxt, ok, cur_job;
  if (threadIdx.x == 0) {
    cur_job = -1;
    nxt = atomicAdd(&st->next, 1);
  }
  while (true) {
    if (threadIdx.x == 0) {
      const int k = ld_acquire(&st->abort) ? nwork : nxt;
      item = k;
      ok = 1;
      if (k < nwork) {
        const PWork w = work[k];
        if (w.w0 >= 0) ok = wait_count(&st->cnt[w.w0], w.n0, st, limit_ns);
        if (ok && w.w1 >= 0) ok = wait_count(&st->cnt[w.w1], w.n1, st, limit_ns);
        // claim the next item now, while this one runs. (Claiming two ahead and
        // prefetching descriptors measured slower on GB300: it hoards the last
        // items on busy CTAs and raises register spills.)
        nxt = ok ? atomicAdd(&st->next, 1) : nwork;
      }
    }
    __syncthreads();
    const int k = item;
    if (k >= nwork || !ok) break;
    const PWork w = work[k];
    if (w.job != cur_job) {
      // the job's descriptor into shared memory (read by every tile body)
      const int *src = reinterpret_cast<const int *>(jobs + w.job);
      int *dst = reinterpret_cast<int *>(&J);
      for (int q = threadIdx.x; q < (int)(sizeof(PJob) / sizeof(int)); q += kPNT) dst[q] = src[q];
      __syncthreads();
      if (threadIdx.x == 0) cur_job = w.job;
    }
    switch (J.logn) {
      case 13: run_stage<13>(J, w.stage, w.bx, w.by, raw, cst); break;
      case 14: run_stage<14>(J, w.stage, w.bx, w.by, raw, cst); break;
      case 15: run_stage<15>(J, w.stage, w.bx, w.by, raw, cst); break;
      case 16: run_stage<16>(J, w.stage, w.bx, w.by, raw, cst); break;
      default: run_stage<17>(J, w.stage, w.bx, w.by, raw, cst); break;
    }
    __syncthreads();
    if (threadIdx.x == 0 && w.sig >= 0) red_release_add(&st->cnt[w.sig], 1);
  }
}

constexpr int cmax_(int a, int b) { return a > b ? a : b; }

// Stage-major form: one persistent kernel per stage over every job's tiles of that
// stage, the kernels chained by programmatic dependent launch (each tile body waits for
// the previous stage's kernel before it reads a buffer another stage wrote). A stage
// has no dependencies inside itself, so its CTAs only claim items: no waits. Each
// stage kernel holds one stage body per N (its own register budget) and its own block
// size: 256 threads for the column passes (tiles of 2^10 points at radix 4, 2^11 at
// radix 8), 128 for the row passes (2^9 at radix 4, 2^10 at radix 8).
// CLS: the key multiply and the ModDown row pass (stages 3 and 7) run in two launches,
// N <= 2^15 (CLS 1: 2^9-point row tiles, 128 threads) and N >= 2^16 (CLS 2: 2^10-point
// row tiles, 256 threads), both with the software-pipelined radix-4 bodies; every other
// stage is one launch (CLS 0).
template <int S, int CLS = 0>
struct SCfg {
  static constexpr bool ROW = S == 0 || S == 3 || S == 4 || S == 7;
  static constexpr bool PIPE = S == 3 || S == 7;
  static constexpr int NT = PIPE ? (CLS == 2 ? 256 : 128) : ROW ? 128 : 256;
  // resident blocks per SM (register budget): 64 registers, except the basis-conversion
  // column passes (80), which spill at 64
  static constexpr int MINB = S == 2 || S == 6 ? 3 : 1024 / NT;
  static constexpr int LO = CLS == 2 ? 16 : 13, HI = CLS == 1 ? 15 : 17;  // log N range
};
__host__ __device__ constexpr int srl_row(int logn) { return geo_tile_log_row(logn) - 7; }

template <int LOGN, int S>
__device__ __forceinline__ void sstage(const PJob &J, int bx, int by, unsigned char *raw,
                                       u64 *cst) {
  constexpr int RC = prl_col(LOGN), RR = srl_row(LOGN);
  static_assert(kern::ROW_PIPE<LOGN, 2>, "pipelined row bodies at two-pass sizes");
  if constexpr (S == 0) kern::inv_row_body<LOGN, RR>(J.a, J.jp, J.wo, 0, bx, by, raw);
  if constexpr (S == 1) kern::inv_col_body<LOGN, RC, 0>(J.a, J.jp, J.wo, 0, bx, by, raw);
  if constexpr (S == 2)
    kern::fwd_col_body<LOGN, RC, kern::PRO_UP, 0>(J.a, J.jp, J.wo, J.up, BUF_TMP, bx, by, raw,
                                                  cst);
  if constexpr (S == 3) kern::keymult_pipe_body<LOGN, 2>(J.a, J.jp, J.wo, J.tg, bx, by, raw);
  if constexpr (S == 4) kern::inv_row_body<LOGN, RR>(J.a, J.jp, J.wo, 1, bx, by, raw);
  if constexpr (S == 5) kern::inv_col_body<LOGN, RC, 0>(J.a, J.jp, J.wo, 1, bx, by, raw);
  if constexpr (S == 6)
    kern::fwd_col_body<LOGN, RC, kern::PRO_DOWN, 0>(J.a, J.jp, J.wo, J.dn, BUF_TMP2, bx, by, raw,
                                                    cst);
  if constexpr (S == 7) kern::moddown_pipe_body<LOGN, 2>(J.a, J.jp, J.wo, J.d1, bx, by, raw);
}

// Items [off, off + n) of the work list (all of stage S, of class CLS), claimed one at a
// time through counter st->snext[ctr].
template <int S, int CLS>
__global__ void __launch_bounds__(SCfg<S, CLS>::NT, SCfg<S, CLS>::MINB)
    k_pstage(const PJob *__restrict__ jobs, const PWork *__restrict__ work, int off, int n,
             PState *st, int ctr) {
  using C = SCfg<S, CLS>;
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ u64 cst[kMaxLimbs];
  __shared__ PJob J;
  __shared__ int item, cur_job;
  if (threadIdx.x == 0) cur_job = -1;
  while (true) {
    if (threadIdx.x == 0) item = atomicAdd(&st->snext[ctr], 1);
    __syncthreads();
    const int k = item;
    if (k >= n) break;
    const PWork w = work[off + k];
    if (w.job != cur_job) {
      const int *src = reinterpret_cast<const int *>(jobs + w.job);
      int *dst = reinterpret_cast<int *>(&J);
      for (int q = threadIdx.x; q < (int)(sizeof(PJob) / sizeof(int)); q += C::NT) dst[q] = src[q];
      __syncthreads();
      if (threadIdx.x == 0) cur_job = w.job;
    }
    if constexpr (C::LO == 16) {
      if (J.logn == 16)
        sstage<16, S>(J, w.bx, w.by, raw, cst);
      else
        sstage<17, S>(J, w.bx, w.by, raw, cst);
    } else if constexpr (C::HI == 15) {
      switch (J.logn) {
        case 13: sstage<13, S>(J, w.bx, w.by, raw, cst); break;
        case 14: sstage<14, S>(J, w.bx, w.by, raw, cst); break;
        default: sstage<15, S>(J, w.bx, w.by, raw, cst); break;
      }
    } else {
      switch (J.logn) {
        case 13: sstage<13, S>(J, w.bx, w.by, raw, cst); break;
        case 14: sstage<14, S>(J, w.bx, w.by, raw, cst); break;
        case 15: sstage<15, S>(J, w.bx, w.by, raw, cst); break;
        case 16: sstage<16, S>(J, w.bx, w.by, raw, cst); break;
        default: sstage<17, S>(J, w.bx, w.by, raw, cst); break;
      }
    }
    // this tile's generic shared-memory reads before the next tile's bulk copies
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  pdl_trigger();
}

template <int S, int LOGN>
constexpr int ssmem_one() {
  using GR = GeoT<LOGN, 2, 1>;
  return S == 3   ? kern::KmSmem<GR>::BYTES
         : S == 7 ? kern::MdSmem<GR>::BYTES
         : SCfg<S>::ROW ? GeoT<LOGN, srl_row(LOGN), 1>::SMEM_ROW
                        : GeoT<LOGN, prl_col(LOGN), 0>::SMEM_COL;
}
template <int S, int CLS>
constexpr int ssmem() {
  int m = 0;
  for (int l = SCfg<S, CLS>::LO; l <= SCfg<S, CLS>::HI; ++l) {
    const int v = l == 13   ? ssmem_one<S, 13>()
                  : l == 14 ? ssmem_one<S, 14>()
                  : l == 15 ? ssmem_one<S, 15>()
                  : l == 16 ? ssmem_one<S, 16>()
                            : ssmem_one<S, 17>();
    m = cmax_(m, v);
  }
  return m;
}
template <int LOGN>
constexpr bool snt_ok() {
  return GeoT<LOGN, srl_row(LOGN), 1>::NT == 128 && GeoT<LOGN, prl_col(LOGN), 0>::NT == 256 &&
         GeoT<LOGN, 2, 1>::NT == (LOGN >= 16 ? 256 : 128);
}
static_assert(snt_ok<13>() && snt_ok<14>() && snt_ok<15>() && snt_ok<16>() && snt_ok<17>(),
              "one block size per pass kind");

template <int LOGN>
constexpr int smem_of() {
  using GC = GeoT<LOGN, prl_col(LOGN), 0>;
  using GR = GeoT<LOGN, prl_row(LOGN), 1>;
  return GC::SMEM_COL > GR::SMEM_ROW ? GC::SMEM_COL : GR::SMEM_ROW;
}
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kPSmem =
    cmax(cmax(cmax(smem_of<13>(), smem_of<14>()), cmax(smem_of<15>(), smem_of<16>())),
         smem_of<17>());

template <int LOGN>
constexpr bool nt_ok() {
  return GeoT<LOGN, prl_col(LOGN), 0>::NT == kPNT && GeoT<LOGN, prl_row(LOGN), 1>::NT == kPNT;
}
static_assert(nt_ok<13>() && nt_ok<14>() && nt_ok<15>() && nt_ok<16>() && nt_ok<17>(),
              "one block size for every size and pass");

int grid_of(int logn, int which) {
  // column-pass grid (which 1) or row-pass grid (which 0) for N = 2^logn
  const int loga = geo_loga(logn), logb = logn - loga;
  const int gc = 1 << (geo_tile_log_col(logn) - loga), gr = 1 << (geo_tile_log_row(logn) - logb);
  return which ? (1 << logb) / gc : (1 << loga) / gr;
}

}  // namespace

// Host side of the persistent batch (called by ks_switch_batch).
struct PersistBatch {
  std::vector<PJob> jobs;
  std::vector<PWork> work;
  int ncnt = 0;
  int soff[kStages + 1] = {};  // work[soff[s] .. soff[s + 1]) is stage s
  int big_end[kStages] = {};    // stages 3 and 7: items of N >= 2^16 jobs first, up to here
};

// kStages + 1 stage boundaries, then the ends of stage 3's and stage 7's N >= 2^16 items.
void persist_stage_offsets(const PersistBatch &pb, int *off) {
  for (int s = 0; s <= kStages; ++s) off[s] = pb.soff[s];
  off[kStages + 1] = pb.big_end[3];
  off[kStages + 2] = pb.big_end[7];
}

bool persist_supported(const ks_context *c) { return c->logn >= 13 && c->logn <= 17; }

PersistBatch *persist_new() { return new PersistBatch(); }
void persist_free(PersistBatch *pb) { delete pb; }
int persist_counts(const PersistBatch &pb, int *njobs, int *nwork, int *ncnt) {
  *njobs = (int)pb.jobs.size();
  *nwork = (int)pb.work.size();
  *ncnt = pb.ncnt;
  return KS_OK;
}

int persist_radix(int logn) { return prl_col(logn); }

namespace {

// Counter layout of one job (offsets into PState::cnt).
struct JobCounters {
  int c01;  // [nq]          row tiles of limb i done (stage 0)
  int c12;  // [beta][gc]    limbs of digit j done in col tile c (stage 1)
  int c23;  // [qp]          (col tile, digit) items of target t done (stage 2)
  int c3p;  // [np][gr]      key multiply of P-target k, row tile r (stage 3)
  int c3q;  // [nq][gr]      key multiply of Q-target i, row tile r (stage 3)
  int c45;  // [np]          row tiles of P-limb k done (stage 4)
  int c56;  // [gc]          P-limbs done in col tile c (stage 5)
  int c67;  // [nq]          (col tile, c) items of limb i done (stage 6)
};

}  // namespace

// Build the descriptors, counters and the stage-major work list for jobs whose
// plans are DPOB fused (OutputBulk: one group per phase).
void persist_build(PersistBatch &pb, const std::vector<const ks_context *> &ctx,
                   const std::vector<JobPtr> &jp, const std::vector<WsOff> &wo) {
  pb.jobs.clear();
  pb.work.clear();
  pb.ncnt = 0;
  const int n = (int)ctx.size();
  std::vector<JobCounters> jc(n);
  std::vector<long long> work(n);
  for (int k = 0; k < n; ++k) {
    const ks_context *c = ctx[k];
    PJob J;
    std::memset(&J, 0, sizeof(J));
    J.a = kern::make_args(c);
    J.jp = jp[k];
    J.wo = wo[k];
    J.logn = c->logn;
    Tasks up = {};
    up.mode = TASK_UP;
    up.t0 = 0;
    up.t1 = c->qp;
    up.j0 = 0;
    up.j1 = c->beta;
    up.sm.sj = c->qp;
    up.sm.st = 1;
    up.sm.base = 0;
    up.first = 1;
    Tasks tg = up;
    tg.mode = TASK_TARGET;
    Tasks dn = {};
    dn.mode = TASK_DOWN;
    dn.i0 = 0;
    dn.i1 = c->nq;
    dn.span = c->nq;
    dn.ibase = 0;
    Tasks d1 = dn;
    d1.mode = TASK_DOWN1;
    J.up = up;
    J.tg = tg;
    J.dn = dn;
    J.d1 = d1;
    pb.jobs.push_back(J);
    const int gr = grid_of(c->logn, 0), gc = grid_of(c->logn, 1);
    JobCounters &q = jc[k];
    int o = pb.ncnt;
    q.c01 = o; o += c->nq;
    q.c12 = o; o += c->beta * gc;
    q.c23 = o; o += c->qp;
    q.c3p = o; o += c->np * gr;
    q.c3q = o; o += c->nq * gr;
    q.c45 = o; o += c->np;
    q.c56 = o; o += gc;
    q.c67 = o; o += c->nq;
    pb.ncnt = o;
    work[k] = (long long)(c->qp * c->beta) << c->logn;
  }
  // largest jobs first within each stage (measured 1% faster than batch order)
  std::vector<int> ord(n);
  for (int k = 0; k < n; ++k) ord[k] = k;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return work[x] > work[y]; });
  auto item = [&](int k, int s, int bx, int by, int w0, int n0, int w1, int n1, int sig) {
    PWork w;
    w.job = (uint16_t)k;
    w.bx = (uint16_t)bx;
    w.by = (uint16_t)by;
    w.stage = (uint8_t)s;
    w.pad = 0;
    w.w0 = w0;
    w.n0 = (uint16_t)n0;
    w.w1 = w1;
    w.n1 = (uint16_t)n1;
    w.sig = sig;
    pb.work.push_back(w);
  };
  for (int s = 0; s < kStages; ++s) {
    pb.soff[s] = (int)pb.work.size();
    for (int kk = 0; kk < n; ++kk) {
      const int k = ord[kk];
      const ks_context *c = ctx[k];
      const PJob &J = pb.jobs[k];
      const JobCounters &q = jc[k];
      const int gr = grid_of(c->logn, 0), gc = grid_of(c->logn, 1);
      const int nq = c->nq, np = c->np, al = c->alpha;
      auto dsize = [&](int j) { return std::min(nq, (j + 1) * al) - j * al; };
      auto ndig = [&](int t) { return c->beta - (t < nq ? 1 : 0); };
      switch (s) {
        case 0:
          for (int i = 0; i < nq; ++i)
            for (int r = 0; r < gr; ++r) item(k, 0, r, i, -1, 0, -1, 0, q.c01 + i);
          break;
        case 1:
          for (int i = 0; i < nq; ++i)
            for (int cc = 0; cc < gc; ++cc)
              item(k, 1, cc, i, q.c01 + i, gr, -1, 0, q.c12 + (i / al) * gc + cc);
          break;
        case 2: {
          const int nt = kern::count_tasks(c, J.up);
          for (int y = 0; y < nt; ++y) {
            const uint32_t w = kern::decode(J.a, J.up, y);
            const int t = task_limb(w), j = task_dig(w);
            for (int cc = 0; cc < gc; ++cc)
              item(k, 2, cc, y, q.c12 + j * gc + cc, dsize(j), -1, 0, q.c23 + t);
          }
          break;
        }
        case 3:
          for (int t = 0; t < c->qp; ++t)
            for (int r = 0; r < gr; ++r)
              item(k, 3, r, t, ndig(t) > 0 ? q.c23 + t : -1, gc * ndig(t), -1, 0,
                   t < nq ? q.c3q + t * gr + r : q.c3p + (t - nq) * gr + r);
          break;
        case 4:
          for (int kp = 0; kp < np; ++kp)
            for (int r = 0; r < gr; ++r)
              item(k, 4, r, kp, q.c3p + kp * gr + r, 1, -1, 0, q.c45 + kp);
          break;
        case 5:
          for (int kp = 0; kp < np; ++kp)
            for (int cc = 0; cc < gc; ++cc) item(k, 5, cc, kp, q.c45 + kp, gr, -1, 0, q.c56 + cc);
          break;
        case 6: {
          const int nt = kern::count_tasks(c, J.dn);
          for (int y = 0; y < nt; ++y) {
            const int i = task_limb(kern::decode(J.a, J.dn, y));
            for (int cc = 0; cc < gc; ++cc) item(k, 6, cc, y, q.c56 + cc, np, -1, 0, q.c67 + i);
          }
          break;
        }
        default:
          for (int i = 0; i < nq; ++i)
            for (int r = 0; r < gr; ++r)
              item(k, 7, r, i, q.c67 + i, 2 * gc, q.c3q + i * gr + r, 1, -1);
          break;
      }
    }
  }
  pb.soff[kStages] = (int)pb.work.size();
  // stages 3 and 7 run as two launches by row-tile size: N >= 2^16 items first
  for (int st : {3, 7}) {
    auto b = pb.work.begin() + pb.soff[st], e = pb.work.begin() + pb.soff[st + 1];
    auto mid = std::stable_partition(b, e, [&](const PWork &w) { return pb.jobs[w.job].logn >= 16; });
    pb.big_end[st] = (int)(mid - pb.work.begin());
  }
}

size_t persist_state_bytes(int ncnt) { return sizeof(PState) + sizeof(int) * (size_t)ncnt; }

// Device image of a built batch: jobs | work | state (16-byte aligned pieces).
static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
size_t persist_bytes(const PersistBatch &pb) {
  return align16(pb.jobs.size() * sizeof(PJob)) + align16(pb.work.size() * sizeof(PWork)) +
         persist_state_bytes(pb.ncnt);
}
size_t persist_state_offset(const PersistBatch &pb) {
  return align16(pb.jobs.size() * sizeof(PJob)) + align16(pb.work.size() * sizeof(PWork));
}

// Copy the descriptors and the work list to `dev` (stream-ordered; not capturable:
// done before any capture).
int persist_upload(const PersistBatch &pb, void *dev, cudaStream_t s) {
  const size_t jb = pb.jobs.size() * sizeof(PJob), wb = pb.work.size() * sizeof(PWork);
  cudaError_t e = cudaMemcpyAsync(dev, pb.jobs.data(), jb, cudaMemcpyHostToDevice, s);
  if (!e)
    e = cudaMemcpyAsync((char *)dev + align16(jb), pb.work.data(), wb, cudaMemcpyHostToDevice, s);
  return e ? KS_ECUDA : KS_OK;
}

// Reset the state and launch the persistent kernel over an uploaded image
// (capturable). `stall` (tests only) starts the first counter at -1, so the items
// that wait on it (job 0's first column items) wait until the bounded wait gives up.
int persist_launch(void *dev, int njobs, int nwork, int ncnt, size_t state_offset,
                   unsigned long long limit_ns, bool stall, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  static int blocks_per_sm = 0, sms = 0;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_persist, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared);
    int d = 0;
    if (attr == cudaSuccess) attr = cudaGetDevice(&d);
    if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
    if (attr == cudaSuccess)
      attr = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_persist, kPNT, kPSmem);
  });
  if (attr != cudaSuccess || blocks_per_sm < 1) return KS_ECUDA;
  char *base = (char *)dev;
  const size_t jb = align16((size_t)njobs * sizeof(PJob));
  PState *st = (PState *)(base + state_offset);
  cudaError_t e = cudaMemsetAsync(st, 0, persist_state_bytes(ncnt), s);
  if (!e && stall) e = cudaMemsetAsync(&st->cnt[0], 0xff, sizeof(int), s);  // -1
  if (e) return KS_ECUDA;
  const int grid = std::max(1, std::min(nwork, blocks_per_sm * sms));
  k_persist<<<grid, kPNT, kPSmem, s>>>((const PJob *)base, (const PWork *)(base + jb), nwork, st,
                                       limit_ns);
  return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ECUDA;
}

namespace {
template <int S, int CLS>
cudaError_t stage_prepare(int *blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_pstage<S, CLS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ssmem<S, CLS>());
  if (!e)
    e = cudaFuncSetAttribute(k_pstage<S, CLS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (!e)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pstage<S, CLS>,
                                                      SCfg<S, CLS>::NT, ssmem<S, CLS>());
  return e;
}
// Items [b, e) of the work list through counter ctr.
template <int S, int CLS>
cudaError_t stage_launch(const PJob *jobs, const PWork *work, int b, int e, int ctr, PState *st,
                         int grid_max, bool first, cudaStream_t s) {
  const int n = e - b;
  if (n == 0) return cudaSuccess;
  const int grid = std::max(1, std::min(n, grid_max));
  if (first) {  // after the state reset: an ordinary dependency
    k_pstage<S, CLS><<<grid, SCfg<S, CLS>::NT, ssmem<S, CLS>(), s>>>(jobs, work, b, n, st, ctr);
    return cudaGetLastError();
  }
  return launch_pdl(k_pstage<S, CLS>, dim3(grid), dim3(SCfg<S, CLS>::NT), ssmem<S, CLS>(), s,
                    jobs, work, b, n, st, ctr);
}
}  // namespace

// Reset the state and launch the stage-major kernels over an uploaded image
// (capturable): ten launches (stages 3 and 7 in two), each waiting for the previous one.
int persist_launch_staged(void *dev, int njobs, const int *off, int ncnt, size_t state_offset,
                          cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  static int bps[kStages + 2] = {}, sms = 0;
  std::call_once(once, [] {
    int d = 0;
    attr = cudaGetDevice(&d);
    if (!attr) attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
    if (!attr) attr = stage_prepare<0, 0>(&bps[0]);
    if (!attr) attr = stage_prepare<1, 0>(&bps[1]);
    if (!attr) attr = stage_prepare<2, 0>(&bps[2]);
    if (!attr) attr = stage_prepare<3, 2>(&bps[3]);
    if (!attr) attr = stage_prepare<3, 1>(&bps[8]);
    if (!attr) attr = stage_prepare<4, 0>(&bps[4]);
    if (!attr) attr = stage_prepare<5, 0>(&bps[5]);
    if (!attr) attr = stage_prepare<6, 0>(&bps[6]);
    if (!attr) attr = stage_prepare<7, 2>(&bps[7]);
    if (!attr) attr = stage_prepare<7, 1>(&bps[9]);
  });
  if (attr != cudaSuccess) return KS_ECUDA;
  for (int k = 0; k < kStages + 2; ++k)
    if (bps[k] < 1) return KS_ECUDA;
  char *base = (char *)dev;
  const PJob *jobs = (const PJob *)base;
  const PWork *work = (const PWork *)(base + align16((size_t)njobs * sizeof(PJob)));
  PState *st = (PState *)(base + state_offset);
  const int e3 = off[kStages + 1], e7 = off[kStages + 2];
  cudaError_t e = cudaMemsetAsync(st, 0, persist_state_bytes(ncnt), s);
  if (!e) e = stage_launch<0, 0>(jobs, work, off[0], off[1], 0, st, bps[0] * sms, true, s);
  if (!e) e = stage_launch<1, 0>(jobs, work, off[1], off[2], 1, st, bps[1] * sms, false, s);
  if (!e) e = stage_launch<2, 0>(jobs, work, off[2], off[3], 2, st, bps[2] * sms, false, s);
  if (!e) e = stage_launch<3, 2>(jobs, work, off[3], e3, 3, st, bps[3] * sms, false, s);
  if (!e) e = stage_launch<3, 1>(jobs, work, e3, off[4], 8, st, bps[8] * sms, false, s);
  if (!e) e = stage_launch<4, 0>(jobs, work, off[4], off[5], 4, st, bps[4] * sms, false, s);
  if (!e) e = stage_launch<5, 0>(jobs, work, off[5], off[6], 5, st, bps[5] * sms, false, s);
  if (!e) e = stage_launch<6, 0>(jobs, work, off[6], off[7], 6, st, bps[6] * sms, false, s);
  if (!e) e = stage_launch<7, 2>(jobs, work, off[7], e7, 7, st, bps[7] * sms, false, s);
  if (!e) e = stage_launch<7, 1>(jobs, work, e7, off[8], 9, st, bps[9] * sms, false, s);
  return e == cudaSuccess ? KS_OK : KS_ECUDA;
}

// Error word of a persistent launch whose state is at dev + state_offset (synchronizes s).
int persist_status(const void *dev, size_t state_offset, cudaStream_t s) {
  int err = 0;
  const PState *st = (const PState *)((const char *)dev + state_offset);
  if (cudaMemcpyAsync(&err, &st->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return KS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return KS_ECUDA;
  return err ? KS_ETIMEOUT : KS_OK;
}

}  // namespace ks
