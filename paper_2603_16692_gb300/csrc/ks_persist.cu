// One persistent launch for a batch of KeySwitches of uneven (dnum, N, L).
//
// Every CTA of a co-resident grid loops: it claims the next work item from a
// device counter, waits until the item's job has finished the previous stage,
// runs the item (one tile of one stage, the same device code as the per-stage
// kernels) and counts it done. Work items are listed stage-major over all jobs
// (every job's stage s before any job's stage s+1), so an item only waits for
// items with smaller indices. Items are claimed in index order, and only by CTAs
// that are running, so the earliest unfinished item is held by a running CTA
// and has nothing left to wait for: the loop cannot deadlock, resident grid or
// not.
//
// Stages of one job (DPOB, fused, two-pass NTT; N = 2^13..2^17):
//   0 iNTT rows (d)   1 iNTT columns (d)   2 ModUp BConv + NTT columns
//   3 NTT rows + key multiply   4 iNTT rows (P-limbs)   5 iNTT columns (P-limbs)
//   6 ModDown BConv + NTT columns   7 NTT rows + P^-1 scaling
//
// Each CTA claims its next item while it runs the current one; a claimed item
// only waits for items with smaller indices, so the argument above still holds.
// Completion is counted with a release increment after the CTA's barrier, and the
// consumer's acquire load of the counter (then a barrier) orders its reads after
// the producer's writes.
//
// Waits are bounded: a wait that exceeds `limit_ns` of %globaltimer sets the
// device error word and the abort flag, and every CTA then returns; the host
// reads the error with ks_batch_status (KS_ETIMEOUT). Buffers written during the
// launch are read with coherent loads after an acquire on the stage counter.
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

// The radix of the rounds for each N: 256 threads per tile at every size.
__host__ __device__ constexpr int prl(int logn) { return logn <= 14 ? 2 : 3; }

struct PJob {
  KArgs a;
  JobPtr jp;
  WsOff wo;
  Tasks up, tg, dn, d1;
  int logn;
  int count[kStages];  // work items of each stage
};

struct PWork {
  uint16_t job;
  uint8_t stage;
  uint8_t pad;
  uint16_t bx, by;
};

struct PState {
  int next;
  int abort;
  int err;
  int pad;
  int done[1];  // [njobs][kStages]
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
  constexpr int RL = prl(LOGN);
  if constexpr (STAGE == 0) kern::inv_row_body<LOGN, RL>(J.a, J.jp, J.wo, which, bx, by, raw);
  if constexpr (STAGE == 1) kern::inv_col_body<LOGN, RL>(J.a, J.jp, J.wo, which, bx, by, raw);
  if constexpr (STAGE == 2)
    kern::fwd_col_body<LOGN, RL, kern::PRO_UP>(J.a, J.jp, J.wo, J.up, BUF_TMP, bx, by, raw, cst);
  if constexpr (STAGE == 3)
    kern::keymult_body<LOGN, RL, kern::PRO_LOAD>(J.a, J.jp, J.wo, J.tg, bx, by, raw, cst);
  if constexpr (STAGE == 6)
    kern::fwd_col_body<LOGN, RL, kern::PRO_DOWN>(J.a, J.jp, J.wo, J.dn, BUF_TMP2, bx, by, raw,
                                                cst);
  if constexpr (STAGE == 7)
    kern::moddown_body<LOGN, RL, kern::PRO_LOAD>(J.a, J.jp, J.wo, J.d1, bx, by, raw, cst);
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
        if (w.stage > 0)
          ok = wait_count(&st->done[w.job * kStages + w.stage - 1],
                          jobs[w.job].count[w.stage - 1], st, limit_ns);
        // claim the next item now, so that the claim's latency hides behind this one
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
    if (threadIdx.x == 0) red_release_add(&st->done[w.job * kStages + w.stage], 1);
  }
}

template <int LOGN>
constexpr int smem_of() {
  using GT = GeoT<LOGN, prl(LOGN)>;
  return GT::SMEM_COL > GT::SMEM_ROW ? GT::SMEM_COL : GT::SMEM_ROW;
}
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kPSmem =
    cmax(cmax(cmax(smem_of<13>(), smem_of<14>()), cmax(smem_of<15>(), smem_of<16>())),
         smem_of<17>());

static_assert(GeoT<13, prl(13)>::NT == kPNT && GeoT<14, prl(14)>::NT == kPNT &&
                  GeoT<15, prl(15)>::NT == kPNT && GeoT<16, prl(16)>::NT == kPNT &&
                  GeoT<17, prl(17)>::NT == kPNT,
              "one block size for every size");

int grid_of(int logn, int which) {
  // column-pass grid (which 1) or row-pass grid (which 0) for N = 2^logn
  const int loga = geo_loga(logn), logb = logn - loga, tl = geo_tile_log(logn);
  const int gc = 1 << (tl - loga), gr = 1 << (tl - logb);
  return which ? (1 << logb) / gc : (1 << loga) / gr;
}

}  // namespace

// Host side of the persistent batch (called by ks_switch_batch).
struct PersistBatch {
  std::vector<PJob> jobs;
  std::vector<PWork> work;
};

bool persist_supported(const ks_context *c) { return c->logn >= 13 && c->logn <= 17; }

PersistBatch *persist_new() { return new PersistBatch(); }
void persist_free(PersistBatch *pb) { delete pb; }
int persist_counts(const PersistBatch &pb, int *njobs, int *nwork) {
  *njobs = (int)pb.jobs.size();
  *nwork = (int)pb.work.size();
  return KS_OK;
}

int persist_radix(int logn) { return prl(logn); }

// Build the descriptors and the stage-major work list for jobs whose plans are
// DPOB fused (OutputBulk: one group per phase).
void persist_build(PersistBatch &pb, const std::vector<const ks_context *> &ctx,
                   const std::vector<JobPtr> &jp, const std::vector<WsOff> &wo) {
  pb.jobs.clear();
  pb.work.clear();
  const int n = (int)ctx.size();
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
    const int gr = grid_of(c->logn, 0), gc = grid_of(c->logn, 1);
    const int items[kStages][2] = {{gr, c->nq},
                                   {gc, c->nq},
                                   {gc, kern::count_tasks(c, up)},
                                   {gr, kern::count_tasks(c, tg)},
                                   {gr, c->np},
                                   {gc, c->np},
                                   {gc, kern::count_tasks(c, dn)},
                                   {gr, kern::count_tasks(c, d1)}};
    for (int s = 0; s < kStages; ++s) J.count[s] = items[s][0] * items[s][1];
    pb.jobs.push_back(J);
  }
  // largest jobs first within each stage (measured 1% faster than batch order)
  std::vector<int> ord(n);
  std::vector<long long> work(n);
  for (int k = 0; k < n; ++k) {
    ord[k] = k;
    work[k] = 0;
    for (int s = 0; s < kStages; ++s) work[k] += pb.jobs[k].count[s];
    work[k] <<= pb.jobs[k].logn;
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return work[x] > work[y]; });
  for (int s = 0; s < kStages; ++s)
    for (int kk = 0; kk < n; ++kk) {
      const int k = ord[kk];
      const PJob &J = pb.jobs[k];
      const int gx = (s == 1 || s == 2 || s == 5 || s == 6) ? grid_of(J.logn, 1)
                                                             : grid_of(J.logn, 0);
      const int gy = J.count[s] / gx;
      for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) {
          PWork w;
          w.job = (uint16_t)k;
          w.stage = (uint8_t)s;
          w.pad = 0;
          w.bx = (uint16_t)bx;
          w.by = (uint16_t)by;
          pb.work.push_back(w);
        }
    }
}

size_t persist_job_bytes() { return sizeof(PJob); }
size_t persist_work_bytes() { return sizeof(PWork); }
size_t persist_state_bytes(int njobs) { return sizeof(PState) + sizeof(int) * (size_t)njobs * kStages; }

// Device image of a built batch: jobs | work | state.
size_t persist_bytes(const PersistBatch &pb) {
  return pb.jobs.size() * sizeof(PJob) + pb.work.size() * sizeof(PWork) +
         persist_state_bytes((int)pb.jobs.size());
}
size_t persist_state_offset(const PersistBatch &pb) {
  return pb.jobs.size() * sizeof(PJob) + pb.work.size() * sizeof(PWork);
}

// Copy the descriptors and the work list to `dev` (stream-ordered; not capturable:
// done before any capture).
int persist_upload(const PersistBatch &pb, void *dev, cudaStream_t s) {
  const size_t jb = pb.jobs.size() * sizeof(PJob), wb = pb.work.size() * sizeof(PWork);
  cudaError_t e = cudaMemcpyAsync(dev, pb.jobs.data(), jb, cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync((char *)dev + jb, pb.work.data(), wb, cudaMemcpyHostToDevice, s);
  return e ? KS_ECUDA : KS_OK;
}

// Reset the state and launch the persistent kernel over an uploaded image
// (capturable). `stall` (tests only) counts job 0's first stage one short, so the
// items of its second stage wait until the bounded wait gives up.
int persist_launch(void *dev, int njobs, int nwork, size_t state_offset,
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
  const size_t jb = (size_t)njobs * sizeof(PJob);
  PState *st = (PState *)(base + state_offset);
  cudaError_t e = cudaMemsetAsync(st, 0, persist_state_bytes(njobs), s);
  if (!e && stall) e = cudaMemsetAsync(&st->done[0], 0xff, sizeof(int), s);  // -1
  if (e) return KS_ECUDA;
  const int grid = std::max(1, std::min(nwork, blocks_per_sm * sms));
  k_persist<<<grid, kPNT, kPSmem, s>>>((const PJob *)base, (const PWork *)(base + jb), nwork, st,
                                       limit_ns);
  return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ECUDA;
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
