// C-ABI of the KeySwitch library: context life cycle, key generation and the
// four dataflows of Sec. III-A (Table III) as launch schedules over the fused
// (or unfused) kernels.
//
//   DSOB  digits one after another; each digit's ModUp + key multiply covers all
//         QP output limbs (footprint O(NL), launches O(dnum)).
//   DPOB  all digits in one launch per step (footprint O(dnum NL), launches O(1)).
//   DSOC  output limbs split into `chunks` groups; per group, digits one after
//         another (footprint O(NL/c), launches O(dnum c)).
//   DPOC  per group, all digits in one launch (footprint O(dnum NL/c), launches O(c)).
// The chunking applies to the QP output limbs of the first phase and to the L+1
// output limbs of the second phase (ModDown); the input iNTT and the iNTT of the
// P-limbs run once in bulk. All variants compute identical bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>

#include "ks_internal.h"
#include "ks_ntt.cuh"

using namespace ks;

namespace {

// Kernel stages whose register-round radix a schedule sets separately.
enum { ST_INV = 0, ST_UPC = 1, ST_KM = 2, ST_DNC = 3, ST_DNR = 4, ST_COUNT = 5 };

struct Plan {
  int base;      // KS_DSOB..KS_DPOC
  bool unfused;
  int rl;        // register-round radix of the plan: 3 (8 points per thread), 2 or 4
  int srl[ST_COUNT];  // per stage (the plan's unless the variant's schedule sets one)
  int ca[ST_COUNT];   // per stage: 1 = alternative column tile (stages with column passes)
  int code;      // every variant bit that changes the launches (graph-cache key)
  bool split;    // KS_SPLIT_DOWN in effect (fused DPOB, two-pass N)
  bool tc_up;    // KS_BCONV_TC in effect (fused, context with a tensor-core path)
  bool tc_down;  // KS_BCONV_TC or KS_BCONV_TC_DOWN in effect
  int chunks;    // phase-1 and phase-2 group counts (1 for OB)
  int clen;      // max QP-limbs per phase-1 group
  int clq;       // max Q-limbs per phase-2 group
  size_t off_v, off_tmp, off_acc, off_vp, off_tmp2, off_pv, off_ppv, total;  // u64 words
  size_t tmp_slots, tmp2_slots;
};

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

constexpr int kSchedMask = 0x3ff << KS_STAGE_SHIFT;

// The tensor-core basis conversions where they measured faster than the integer ones:
// contexts that have them, N >= 2^16 and an input of more than one digit (at
// (4, 2^16, 35) the tuned per-level plans use them at every level with two or more
// digits and at none with one). Added to the plans KS_AUTO takes without a tuned one.
int tc_rule(const ks_context *c) {
  return c->tc_ap > 0 && c->logn >= 16 && c->nq > c->alpha ? KS_BCONV_TC : 0;
}
// The plan a selected context runs: the network's pick (a dataflow and radix among
// integer plans) with the tensor-core rule.
int selected_plan(const ks_context *c) { return c->sel_variant | tc_rule(c); }

int make_plan(const ks_context *c, int variant, int chunks, Plan *pl) {
  if (variant & ~(0xff | KS_UNFUSED | KS_RADIX4 | KS_RADIX16 | kSchedMask | KS_COLTILE_ALT |
                  KS_SPLIT_DOWN | KS_BCONV_TC | KS_BCONV_TC_DOWN))
    return KS_EINVAL;
  if ((variant & KS_RADIX4) && (variant & KS_RADIX16)) return KS_EINVAL;
  if ((variant & 0xff) == KS_AUTO) {
    // the tuned choice for single KeySwitches, else the selector's, else DPOB radix 8
    // (the last two with the tensor-core rule)
    if (c->tuned_variant > 0) {
      variant = c->tuned_variant | (variant & ~0xff);
      if (chunks == 0) chunks = c->tuned_chunks;
    } else if (c->sel_variant > 0) {
      variant = selected_plan(c) | (variant & ~0xff);
      if (chunks == 0) chunks = c->sel_chunks;
    } else {
      variant = KS_DPOB | tc_rule(c) | (variant & ~0xff);
    }
  }
  const int base = variant & 0xff;
  if (base < KS_DSOB || base > KS_DPOC) return KS_EINVAL;
  const bool oc = base == KS_DSOC || base == KS_DPOC;
  if (oc) {
    if (chunks == 0) chunks = 2;
    if (chunks < 1 || chunks > 64) return KS_EINVAL;
  } else {
    chunks = 1;
  }
  pl->base = base;
  pl->unfused = (variant & KS_UNFUSED) != 0;
  pl->rl = (variant & KS_RADIX4) ? 2 : (variant & KS_RADIX16) ? 4 : 3;
  for (int st = 0; st < ST_COUNT; ++st) {
    const int code = (variant >> (KS_STAGE_SHIFT + 2 * st)) & 3;  // 0: the plan's radix
    pl->srl[st] = code == 0 ? pl->rl : code + 1;
  }
  for (int st = 0; st < ST_COUNT; ++st) pl->ca[st] = 0;
  pl->ca[ST_INV] = (variant & KS_COLALT_INV) ? 1 : 0;
  pl->ca[ST_UPC] = (variant & KS_COLALT_UPC) ? 1 : 0;
  pl->ca[ST_DNC] = (variant & KS_COLALT_DNC) ? 1 : 0;
  pl->code = variant & ~0xff;
  pl->split = (variant & KS_SPLIT_DOWN) && base == KS_DPOB && !pl->unfused && c->loga > 0;
  pl->tc_up = (variant & KS_BCONV_TC) && !pl->unfused && c->tc_ap > 0;
  pl->tc_down = (variant & (KS_BCONV_TC | KS_BCONV_TC_DOWN)) && !pl->unfused && c->tc_ap > 0;
  pl->chunks = chunks;
  pl->clen = (c->qp + chunks - 1) / chunks;
  pl->clq = (c->nq + chunks - 1) / chunks;
  const bool dp = base == KS_DPOB || base == KS_DPOC;
  const size_t N = c->N;
  size_t slots;
  if (base == KS_DPOB)
    slots = (size_t)c->beta * c->qp;
  else if (base == KS_DSOB)
    slots = c->qp;
  else
    slots = (dp ? (size_t)c->beta : 1) * pl->clen;
  pl->tmp_slots = slots;
  pl->tmp2_slots = 2 * (size_t)(oc ? pl->clq : c->nq);
  size_t off = 0;
  auto take = [&](size_t words) {
    size_t o = off;
    off += (words + 31) / 32 * 32;  // 256-byte aligned pieces
    return o;
  };
  pl->off_v = take((size_t)c->nq * N);
  pl->off_tmp = take(slots * N);
  pl->off_acc = take((size_t)2 * c->qp * N);
  pl->off_vp = take((size_t)2 * c->np * N);
  pl->off_tmp2 = take(pl->tmp2_slots * N);
  // the bf16 bytes of v and vp (16 bytes per residue) for the tensor-core conversions
  pl->off_pv = pl->tc_up ? take((size_t)2 * c->nq * N) : 0;
  pl->off_ppv = pl->tc_down ? take((size_t)4 * c->np * N) : 0;
  pl->total = off;
  return KS_OK;
}

thread_local cudaError_t g_last_cuda = cudaSuccess;

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return KS_OK;
  g_last_cuda = e;
  if (e == cudaErrorMemoryAllocation) return KS_ENOMEM;
  return KS_ECUDA;
}

#define KS_TRY(x)                       \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return cuda_rc(e_); \
  } while (0)

// ---------------------------------------------------------------------------
// Optional per-launch event timing (ks_profile_begin / ks_profile_end).

struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
  double bytes, ops, macs, tflops;
};

struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

thread_local Profiler g_prof;

// Run one launcher; when profiling, bracket it with events on its stream. tflops: the
// launch's tensor-core FLOPs (2 per bf16 multiply-add).
template <class F>
cudaError_t timed(const char *name, double bytes, double ops, double macs, cudaStream_t s,
                  F f, double tflops = 0) {
  if (!g_prof.on) return f();
  cudaEvent_t a = g_prof.get(), b = g_prof.get();
  cudaEventRecord(a, s);
  cudaError_t e = f();
  cudaEventRecord(b, s);
  g_prof.recs.push_back({name, a, b, bytes, ops, macs, tflops});
  return e;
}

int run_plan(ks_context *c, const Plan &pl, const JobSet &js, cudaStream_t s,
             bool allow_split = true) {
  if (js.n == 0) return KS_OK;
  // KS_SPLIT_DOWN: the fork / join below must not interleave with another call's
  const bool split = pl.split && allow_split && c->side;
  std::unique_lock<std::mutex> side_lock(c->side_mu, std::defer_lock);
  if (split) side_lock.lock();
  const size_t N = c->N;
  const double J = js.n;                                 // jobs per launch
  const double W = (double)N * 8 * J;                    // bytes per limb, all jobs
  const double BF_A = (double)N / 2 * c->loga * J;       // butterflies, column pass
  const double BF_B = (double)N / 2 * c->logb * J;       // butterflies, row pass
  const double NJ = (double)N * J;
  const bool single = c->loga == 0;
  auto stage = [&](int st) -> const LaunchTable & {
    return *c->ltab[pl.srl[st] - 2][pl.ca[st]];
  };
  const LaunchTable &L = stage(ST_INV), &LU = stage(ST_UPC), &LK = stage(ST_KM),
                    &LDC = stage(ST_DNC), &LDR = stage(ST_DNR);
  WsOff wo;
  wo.v = (long long)pl.off_v;
  wo.tmp = (long long)pl.off_tmp;
  wo.acc = (long long)pl.off_acc;
  wo.vp = (long long)pl.off_vp;
  wo.tmp2 = (long long)pl.off_tmp2;
  wo.pv = (long long)pl.off_pv;
  wo.ppv = (long long)pl.off_ppv;
  const bool dp = pl.base == KS_DPOB || pl.base == KS_DPOC;
  const bool oc = pl.base == KS_DSOC || pl.base == KS_DPOC;
  auto dsize = [&](int j) { return std::min(c->nq, (j + 1) * c->alpha) - j * c->alpha; };

  // Input iNTT, fused with the per-limb factor N^-1 * Qhat_{j,i}^-1 of the ModUp BConv.
  {
    const double nl = c->nq;
    KS_TRY(timed("intt_row(d)", 2 * nl * W, nl * (BF_B + (single ? NJ : 0)), 0, s,
                 [&] { return L.intt_row(c, js, wo, 0, s); }));
    if (!single)
      KS_TRY(timed("intt_col(d)", (pl.tc_up ? 3 : 2) * nl * W, nl * (BF_A + NJ), 0, s, [&] {
        return pl.tc_up ? L.intt_col_tc(c, js, wo, 0, s) : L.intt_col(c, js, wo, 0, s);
      }));
  }

  // Phase 1: ModUp (BConv + NTT) and key multiply, per output group.
  for (int ch = 0; ch < pl.chunks; ++ch) {
    const int t0 = ch * pl.clen, t1 = std::min(c->qp, t0 + pl.clen);
    if (t0 >= t1) continue;
    Tasks up = {};
    up.mode = TASK_UP;
    up.t0 = t0;
    up.t1 = t1;
    up.sm.st = 1;
    up.sm.base = oc ? -t0 : 0;
    up.sm.sj = dp ? (oc ? pl.clen : c->qp) : 0;
    const int jstep = dp ? c->beta : 1;
    for (int j0 = 0; j0 < c->beta; j0 += jstep) {
      up.j0 = j0;
      up.j1 = j0 + jstep;
      up.first = j0 == 0 ? 1 : 0;
      Tasks tg = up;
      tg.mode = TASK_TARGET;
      const int nconv = L.count(c, up);
      // tc_tg: the targets the tensor-core form converts (each digit's in groups of
      // kTcTargets)
      double src_b = 0, conv_ops = 0, tc_tg = 0;
      for (int j = up.j0; j < up.j1; ++j) src_b += dsize(j) * W;
      {
        for (int j = up.j0; j < up.j1; ++j) {
          Tasks one = up;
          one.j0 = j;
          one.j1 = j + 1;
          const int cnt = L.count(c, one);
          conv_ops += (double)cnt * NJ * (dsize(j) + 1);
          tc_tg += (cnt + kTcTargets - 1) / kTcTargets * kTcTargets;
        }
      }
      const double nt = t1 - t0, nd = up.j1 - up.j0;
      const double own = nd * nt - nconv;
      if (!pl.unfused) {
        // the tensor-core form reads the sources as bytes (16 per residue), runs the
        // products on the tensor cores (tc_ap * 256 FLOPs per target point) and one REDC
        // per output on the integer pipes
        if (!single && pl.tc_up)
          KS_TRY(timed(
              "modup_col", nconv * W + 2 * src_b, nconv * (NJ + BF_A), nconv * NJ, s,
              [&] { return launch_bconv_tc(c, js, wo, up, true, s); },
              tc_tg * NJ * c->tc_ap * 256));
        else if (!single)
          KS_TRY(timed("modup_col", nconv * W + src_b, conv_ops + nconv * BF_A, conv_ops, s,
                       [&] { return LU.modup_col(c, js, wo, up, s); }));
      } else {
        KS_TRY(timed("bconv_up", nconv * W + src_b, conv_ops, conv_ops, s,
                     [&] { return launch_bconv_up(c, js, wo, up, nconv, s); }));
        if (!single)
          KS_TRY(timed("ntt_col", 2 * nconv * W, nconv * BF_A, 0, s,
                       [&] { return LU.ntt_col(c, js, wo, up, BUF_TMP, s); }));
        KS_TRY(timed("ntt_row", 2 * nconv * W, nconv * BF_B, 0, s,
                     [&] { return LU.ntt_row(c, js, wo, up, BUF_TMP, s); }));
      }
      // key multiply: evk 2 words per (digit, target); ext from tmp (or d on own limbs);
      // acc written (and read when accumulating over digit launches)
      const double km_bytes = (2 * nd * nt + nconv + own + (up.first ? 2 : 4) * nt) * W;
      const double km_ops = 2 * nd * nt * NJ + own * NJ;
      if (!pl.unfused && split) {
        // P-limb targets here; Q-limb targets on the side stream, forked after ModUp and
        // joined before the last ModDown pass (the P-limb chain needs no Q-limb acc)
        const double fq = (double)c->nq / c->qp, fp = 1.0 - fq;
        const double b = km_bytes, o = km_ops + nconv * BF_B, m = km_ops;
        KS_TRY(cudaEventRecord(c->ev_fork, s));
        KS_TRY(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        Tasks tp = tg, tq = tg;
        tp.t0 = c->nq;
        tq.t1 = c->nq;
        KS_TRY(timed("modup_row_keymult", fp * b, fp * o, fp * m, s,
                     [&] { return LK.modup_row(c, js, wo, tp, s); }));
        KS_TRY(timed("modup_row_keymult", fq * b, fq * o, fq * m, c->side,
                     [&] { return LK.modup_row(c, js, wo, tq, c->side); }));
        KS_TRY(cudaEventRecord(c->ev_join, c->side));
      } else if (!pl.unfused) {
        const double b = km_bytes + (single ? src_b - nconv * W : 0);
        const double o = km_ops + nconv * BF_B + (single ? conv_ops : 0);
        const double m = km_ops + (single ? conv_ops : 0);
        KS_TRY(timed("modup_row_keymult", b, o, m, s,
                     [&] { return LK.modup_row(c, js, wo, tg, s); }));
      } else {
        KS_TRY(timed("keymult", km_bytes, km_ops, km_ops, s,
                     [&] { return launch_keymult(c, js, wo, tg, s); }));
      }
    }
  }

  // iNTT of the P-limbs of both accumulators, fused with N^-1 * Phat_k^-1.
  {
    const double nl = 2.0 * c->np;
    KS_TRY(timed("intt_row(accP)", 2 * nl * W, nl * (BF_B + (single ? NJ : 0)), 0, s,
                 [&] { return L.intt_row(c, js, wo, 1, s); }));
    if (!single)
      KS_TRY(timed("intt_col(accP)", (pl.tc_down ? 3 : 2) * nl * W, nl * (BF_A + NJ), 0, s,
                   [&] {
                     return pl.tc_down ? L.intt_col_tc(c, js, wo, 1, s)
                                       : L.intt_col(c, js, wo, 1, s);
                   }));
  }

  // Phase 2: ModDown (BConv P->Q + NTT) and (acc - .) * P^-1, per output group.
  for (int ch = 0; ch < pl.chunks; ++ch) {
    const int i0 = ch * pl.clq, i1 = std::min(c->nq, i0 + pl.clq);
    if (i0 >= i1) continue;
    Tasks dn = {};
    dn.mode = TASK_DOWN;
    dn.i0 = i0;
    dn.i1 = i1;
    dn.span = oc ? pl.clq : c->nq;
    dn.ibase = oc ? i0 : 0;
    Tasks d1 = dn;
    d1.mode = TASK_DOWN1;
    const double n = 2.0 * (i1 - i0), vp_b = 2.0 * c->np * W, conv = n * NJ * (c->np + 1.0);
    if (!pl.unfused) {
      if (!single && pl.tc_down)  // counted as for modup_col
        KS_TRY(timed(
            "moddown_col", n * W + 2 * vp_b, n * (NJ + BF_A), n * NJ, s,
            [&] { return launch_bconv_tc(c, js, wo, dn, false, s); },
            2.0 * ((i1 - i0 + kTcTargets - 1) / kTcTargets * kTcTargets) * NJ * c->tc_ap *
                256));
      else if (!single)
        KS_TRY(timed("moddown_col", n * W + vp_b, conv + n * BF_A, conv, s,
                     [&] { return LDC.moddown_col(c, js, wo, dn, s); }));
      const double b = 3 * n * W + (single ? vp_b - n * W : 0);
      const double o = n * (BF_B + NJ) + (single ? conv : 0);
      if (split) KS_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
      KS_TRY(timed("moddown_row", b, o, single ? conv : 0, s,
                   [&] { return LDR.moddown_row(c, js, wo, d1, s); }));
    } else {
      KS_TRY(timed("bconv_down", n * W + vp_b, conv, conv, s,
                   [&] { return launch_bconv_down(c, js, wo, dn, (int)n, s); }));
      if (!single)
        KS_TRY(timed("ntt_col", 2 * n * W, n * BF_A, 0, s,
                     [&] { return LDC.ntt_col(c, js, wo, dn, BUF_TMP2, s); }));
      KS_TRY(timed("ntt_row", 2 * n * W, n * BF_B, 0, s,
                   [&] { return LDR.ntt_row(c, js, wo, dn, BUF_TMP2, s); }));
      KS_TRY(timed("moddown_scale", 3 * n * W, n * NJ, 0, s,
                   [&] { return launch_moddown_scale(c, js, wo, dn, (int)n, s); }));
    }
  }
  return KS_OK;
}

// Internal streams of ks_switch_batch.
constexpr int kBatchStreams = 16;

// Shared state of ks_switch_batch: the batch workspace arena, fork streams,
// dependency events and the captured graphs (keyed by the jobs' pointers).
struct BatchState {
  std::mutex mu;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  size_t next_event = 0;
  struct Graph {
    cudaGraphExec_t exec;
    void *buf;          // persistent-batch image owned by this graph (or null)
    size_t state_off;
  };
  std::map<std::vector<uintptr_t>, Graph> graphs;
  void *pbuf = nullptr;  // image of the last non-graph persistent batch
  size_t pbuf_bytes = 0;
  const void *last_state_buf = nullptr;
  size_t last_state_off = 0;
  cudaStream_t stream(int g) {
    const size_t k = (size_t)g % kBatchStreams;
    while (streams.size() <= k) {
      cudaStream_t st = nullptr;
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      streams.push_back(st);
    }
    return streams[k];
  }
  cudaStream_t cap = nullptr;
  cudaStream_t capture_stream() {
    if (!cap) cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    return cap;
  }
  // Launch a graph after the work queued on s, and make s wait for it.
  int launch_ordered(cudaGraphExec_t exec, cudaStream_t s) {
    cudaStream_t c = capture_stream();
    cudaEvent_t before = event(), after = event();
    cudaError_t e = cudaEventRecord(before, s);
    if (!e) e = cudaStreamWaitEvent(c, before, 0);
    if (!e) e = cudaGraphLaunch(exec, c);
    if (!e) e = cudaEventRecord(after, c);
    if (!e) e = cudaStreamWaitEvent(s, after, 0);
    return cuda_rc(e);
  }
  cudaEvent_t event() {
    if (events.size() < 256) {
      cudaEvent_t e = nullptr;
      cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      events.push_back(e);
      return e;
    }
    return events[next_event++ % events.size()];
  }
};

BatchState g_batch;

void clear_graphs_locked() {
  for (auto &kv : g_batch.graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.buf) cudaFree(kv.second.buf);
  }
  g_batch.graphs.clear();
  g_batch.last_state_buf = nullptr;
}

// Drop the captured graphs that use context c (before c is freed).
void forget_graphs(ks_context *c) {
  std::lock_guard<std::mutex> lk(g_batch.mu);
  for (auto it = g_batch.graphs.begin(); it != g_batch.graphs.end();) {
    bool uses = false;
    const size_t nj = it->first.empty() ? 0 : (size_t)it->first[0];
    for (size_t k = 0; k < nj && 2 + 5 * k < it->first.size(); ++k)
      if (it->first[2 + 5 * k] == (uintptr_t)c) uses = true;
    if (uses) {
      cudaGraphExecDestroy(it->second.exec);
      if (it->second.buf) {
        if (g_batch.last_state_buf == it->second.buf) g_batch.last_state_buf = nullptr;
        cudaFree(it->second.buf);
      }
      it = g_batch.graphs.erase(it);
    } else {
      ++it;
    }
  }
}

// A context for Q = q[0..L], P = p[0..alpha); `top` (or null) is the context whose
// keys this one reads (a level view: same P and alpha, key layout of the top level).
int create_context(int dnum, int logn, int L, const u64 *q, const u64 *p, int alpha,
                   const ks_context *top, ks_context **out) {
  const int nq = L + 1;
  const int beta = (nq + alpha - 1) / alpha;
  const int qp = nq + alpha;
  if (qp > kMaxLimbs) return KS_EINVAL;
  std::vector<u64> mods(q, q + nq);
  mods.insert(mods.end(), p, p + alpha);
  const u64 two_n = (u64)2 << logn;
  u64 maxq = 0, maxp = 0, maxm = 0;
  for (int t = 0; t < qp; ++t) {
    const u64 m = mods[t];
    if (m >= ((u64)1 << 62) || m % two_n != 1 || !ks::is_prime_u64(m)) return KS_EPRIME;
    for (int k = 0; k < t; ++k)
      if (mods[k] == m) return KS_EPRIME;
    if (t < nq) maxq = std::max(maxq, m); else maxp = std::max(maxp, m);
    maxm = std::max(maxm, m);
  }
  // Exact 128-bit sums must stay below m 2^64 for one REDC:
  //   key multiply  beta * m^2 < m 2^64  <=>  beta * m < 2^64.
  if ((unsigned __int128)beta * maxm >= ((unsigned __int128)1 << 64)) return KS_EINVAL;
  ks_context *c = new (std::nothrow) ks_context();
  if (!c) return KS_ENOMEM;
  c->dnum = dnum;
  c->logn = logn;
  c->L = L;
  c->alpha = alpha;
  c->beta = beta;
  c->nq = nq;
  c->np = alpha;
  c->qp = qp;
  c->eqp = top ? top->qp : qp;
  c->epb = top ? top->nq : nq;
  c->top_L = top ? top->L : -1;
  c->N = 1 << logn;
  c->loga = ks::geo_loga(logn);
  c->logb = logn - c->loga;
  c->loggr = ks::geo_loggr(logn);
  for (int r = 0; r < 3; ++r)
    for (int ca = 0; ca < 2; ++ca) {
      const LaunchTable *t = ks::launch_table(logn, r + 2, ca);
      if (!t || t->prepare() != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return KS_ECUDA;
      }
      c->ltab[r][ca] = t;
    }
  c->lt = c->ltab[1][0];
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    delete c;
    return KS_ECUDA;
  }
  c->mods = mods;
  // basis-conversion sums: run * max_source * m < m 2^64
  c->run_up = (int)std::min<u64>(1 << 20, (~(u64)0) / maxq);
  c->run_down = (int)std::min<u64>(1 << 20, (~(u64)0) / maxp);
  // Tensor-core basis conversions (ks_tc.cu): two-pass N, 2..9 sources per set (the
  // fp32 sums of byte products stay exact below 2^23 up to 16 sources; the source bytes
  // of a 1024-point tile fill the shared memory at 9), one REDC per sum, at most
  // kTcMaxSets digits.
  if (c->loga > 0 && logn <= 17 && alpha >= 2 && alpha <= 9 && beta <= ks::kTcMaxSets &&
      c->run_up >= alpha && c->run_down >= alpha) {
    c->tc_ap = (alpha + 2) & ~1;  // alpha + 1 slots (the last adds 2^23), rounded to even
    c->tc_tplog = ks::kTcTpLog;   // column tiles of the tensor-core items
    if (ks::tc_prepare(logn) != cudaSuccess) {
      cudaGetLastError();
      c->tc_ap = c->tc_tplog = 0;
    }
  }
  cudaGetDevice(&c->device);
  int rc = ks::build_tables(c);
  if (rc) {
    delete c;
    return rc;
  }
  *out = c;
  return KS_OK;
}

// Key generation for a top-level context: lift, NTT every limb, optionally square
// s_from (relinearisation key), combine.
int keygen_impl(ks_context *c, const int8_t *s_from, const int8_t *s_to, unsigned kinv,
                bool square, const uint64_t *a, const int32_t *e, uint64_t *evk, void *stream) {
  if (!c || !s_from || !s_to || !a || !e || !evk) return KS_EINVAL;
  if (c->top_L >= 0) return KS_EINVAL;  // keys are made at the top level
  if (!aligned16(a) || !aligned16(evk)) return KS_EALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = c->N;
  const int npoly = 2 + c->beta;
  u64 *polys = nullptr;
  if (cudaMalloc(&polys, (size_t)npoly * c->qp * N * 8) != cudaSuccess) {
    cudaGetLastError();
    return KS_ENOMEM;
  }
  int rc = KS_OK;
  do {
    cudaError_t err = launch_keygen_lift(c, s_from, s_to, e, kinv, polys, s);
    if (err) { rc = cuda_rc(err); break; }
    // transform every lifted limb in place
    JobSet js = {};
    js.n = 1;
    js.j[0].ws = polys;
    WsOff wo = {};
    Tasks lin = {};
    lin.mode = TASK_LINEAR;
    lin.n = npoly * c->qp;
    err = c->lt->ntt_col(c, js, wo, lin, BUF_TMP, s);
    if (!err) err = c->lt->ntt_row(c, js, wo, lin, BUF_TMP, s);
    if (!err && square) err = launch_keygen_square(c, polys, s);
    if (err) { rc = cuda_rc(err); break; }
    err = launch_keygen_combine(c, polys, (const u64 *)a, (u64 *)evk, s);
    if (err) { rc = cuda_rc(err); break; }
    err = cudaStreamSynchronize(s);
    if (err) rc = cuda_rc(err);
  } while (0);
  cudaFree(polys);
  return rc;
}

// Device address of a pinned (page-locked, device-mapped) host buffer, or null for
// pageable memory and device memory.
const u64 *host_mapped(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  return (const u64 *)at.devicePointer;
}

// At most this many graphs are kept per context (least recently used dropped).
constexpr size_t kGraphCache = 32;

void drop_graph_cache(ks_context *c) {
  std::lock_guard<std::mutex> lk(c->gmu);
  if (!c->gcache.empty()) cudaDeviceSynchronize();  // no replay of these graphs in flight
  for (auto &kv : c->gcache)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  c->gcache.clear();
}

// Enqueue one operation on s through the context's graph cache: the first call
// with a key runs enqueue(s) directly; the second captures enqueue on a private
// stream into a CUDA graph (the kernel chain then launches without per-kernel
// launch gaps); later calls replay it. While the library profiler is on, every
// call runs directly (per-launch events need the individual launches).
//
// Which operations use it (measured on GB300): the kernels of an operation are
// chained by programmatic dependent launch, which also overlaps consecutive
// operations on a stream when they are launched directly but not across graph
// launches. Directly launched, (2, 2^15, 10) runs at 76.7 us per KeySwitch against
// 83.0 us replayed from graphs. Graphs are used where launches cost more than they
// overlap: single-pass sizes (N <= 2^12, a few microseconds of GPU work per kernel)
// and the synchronous host-buffer entry point (one launch per call).
bool use_graphs(const ks_context *c) { return c->loga == 0; }
template <class F>
int cached_launch(ks_context *c, const std::array<uintptr_t, 10> &key, cudaStream_t s,
                  F enqueue) {
  if (g_prof.on) return enqueue(s);
  std::unique_lock<std::mutex> lk(c->gmu);
  auto it = c->gcache.find(key);
  if (it == c->gcache.end()) {
    if (c->gcache.size() >= kGraphCache) {
      auto old = c->gcache.begin();
      for (auto q = c->gcache.begin(); q != c->gcache.end(); ++q)
        if (q->second.last < old->second.last) old = q;
      if (old->second.exec) cudaGraphExecDestroy(old->second.exec);
      c->gcache.erase(old);
    }
    c->gcache[key].last = ++c->gclock;
    lk.unlock();
    return enqueue(s);
  }
  it->second.last = ++c->gclock;
  if (it->second.direct) {
    lk.unlock();
    return enqueue(s);
  }
  if (!it->second.exec) {
    if (!c->gstream && cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking)) {
      cudaGetLastError();
      lk.unlock();
      return enqueue(s);
    }
    KS_TRY(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(c->gstream);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->gstream, &gr);
    cudaGraphExec_t exec = nullptr;
    if (rc == KS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (rc != KS_OK || e != cudaSuccess || !exec) {
      // not capturable: run this key directly from now on (a real error shows again)
      cudaGetLastError();
      it->second.direct = true;
      lk.unlock();
      return enqueue(s);
    }
    it->second.exec = exec;
  }
  cudaGraphExec_t exec = it->second.exec;
  lk.unlock();
  return cuda_rc(cudaGraphLaunch(exec, s));
}

int plan_code(const Plan &pl) { return pl.base | pl.code; }

// Galois elements are odd residues k in [1, 2N).
bool galois_ok(const ks_context *c, uint32_t k) {
  return (k & 1) && (u64)k < (u64)2 * c->N;
}

// Runs fn(base) on the caller's workspace (if given and large enough) or on the
// context's internal arena (grown as needed; held under its lock while fn enqueues).
template <class F>
int with_workspace(ks_context *c, void *ws, size_t ws_bytes, size_t need, F fn) {
  if (ws) {
    if (ws_bytes < need) return KS_EINVAL;
    return fn((u64 *)ws);
  }
  std::lock_guard<std::mutex> lk(c->ws_mu);
  if (c->ws_bytes < need) {
    if (c->ws) {
      // a smaller arena may still be in use by earlier work on any stream
      cudaDeviceSynchronize();
      cudaFree(c->ws);
      c->ws = nullptr;
      c->ws_bytes = 0;
    }
    if (cudaMalloc(&c->ws, need) != cudaSuccess) {
      cudaGetLastError();
      return KS_ENOMEM;
    }
    c->ws_bytes = need;
  }
  return fn((u64 *)c->ws);
}

// Device-time budget of one wait of the persistent batch kernel.
constexpr unsigned long long kPersistWaitNs = 2000000000ull;

int batch_persistent(const ks_job *jobs, int njobs, int flags, cudaStream_t s) {
  std::vector<const ks_context *> ctxs(njobs);
  std::vector<Plan> plans(njobs);
  size_t total = 0;
  for (int k = 0; k < njobs; ++k) {
    const ks_context *c = jobs[k].ctx;
    if (!persist_supported(c)) return KS_EINVAL;
    ctxs[k] = c;
    const int v = KS_DPOB | (persist_radix(c->logn) == 2 ? KS_RADIX4 : 0);
    int rc = make_plan(c, v, 0, &plans[k]);
    if (rc) return rc;
    total += plans[k].total * 8;
  }
  const bool graph = (flags & KS_BATCH_GRAPH) != 0, stall = (flags & KS_BATCH_TEST_STALL) != 0;
  std::lock_guard<std::mutex> lk(g_batch.mu);
  if (g_batch.arena_bytes < total) {
    if (g_batch.arena) {
      cudaDeviceSynchronize();
      cudaFree(g_batch.arena);
    }
    clear_graphs_locked();
    g_batch.arena = nullptr;
    g_batch.arena_bytes = 0;
    if (cudaMalloc(&g_batch.arena, total) != cudaSuccess) {
      cudaGetLastError();
      return KS_ENOMEM;
    }
    g_batch.arena_bytes = total;
  }
  std::vector<JobPtr> jp(njobs);
  std::vector<WsOff> wo(njobs);
  char *base = (char *)g_batch.arena;
  for (int k = 0; k < njobs; ++k) {
    jp[k].d = (const u64 *)jobs[k].d_dev;
    jp[k].evk = (const u64 *)jobs[k].evk_dev;
    jp[k].out = (u64 *)jobs[k].out_dev;
    jp[k].ws = (u64 *)base;
    base += plans[k].total * 8;
    wo[k] = WsOff{(long long)plans[k].off_v, (long long)plans[k].off_tmp,
                  (long long)plans[k].off_acc, (long long)plans[k].off_vp,
                  (long long)plans[k].off_tmp2};
  }
  std::vector<uintptr_t> key;
  if (graph && !stall) {
    key.push_back((uintptr_t)njobs);
    key.push_back((uintptr_t)s);
    for (int k = 0; k < njobs; ++k) {
      key.push_back((uintptr_t)jobs[k].ctx);
      key.push_back((uintptr_t)jobs[k].d_dev);
      key.push_back((uintptr_t)jobs[k].evk_dev);
      key.push_back((uintptr_t)jobs[k].out_dev);
      key.push_back((uintptr_t)0x7e5157e47ull);  // persistent marker
    }
    auto it = g_batch.graphs.find(key);
    if (it != g_batch.graphs.end()) {
      g_batch.last_state_buf = it->second.buf;
      g_batch.last_state_off = it->second.state_off;
      return g_batch.launch_ordered(it->second.exec, s);
    }
  }
  PersistBatch *pb = persist_new();
  persist_build(*pb, ctxs, jp, wo);
  const size_t bytes = persist_bytes(*pb), soff = persist_state_offset(*pb);
  int nj = 0, nw = 0, nc = 0;
  persist_counts(*pb, &nj, &nw, &nc);
  int stage_off[kPersistStages + 3];
  persist_stage_offsets(*pb, stage_off);
  int rc = KS_OK;
  void *buf = nullptr;
  if (graph && !stall) {
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      persist_free(pb);
      return KS_ENOMEM;
    }
  } else {
    if (g_batch.pbuf_bytes < bytes) {
      if (g_batch.pbuf) {
        cudaDeviceSynchronize();
        cudaFree(g_batch.pbuf);
      }
      g_batch.pbuf = nullptr;
      g_batch.pbuf_bytes = 0;
      if (cudaMalloc(&g_batch.pbuf, bytes) != cudaSuccess) {
        cudaGetLastError();
        persist_free(pb);
        return KS_ENOMEM;
      }
      g_batch.pbuf_bytes = bytes;
    }
    buf = g_batch.pbuf;
  }
  rc = persist_upload(*pb, buf, s);
  persist_free(pb);
  if (rc) return rc;
  // the stage-major kernels; the one-launch dataflow kernel (tile-level dependency
  // counters, bounded waits) for the failure-detection test
  auto launch = [&](cudaStream_t q) {
    return stall ? persist_launch(buf, nj, nw, nc, soff, kPersistWaitNs, true, q)
                 : persist_launch_staged(buf, nj, stage_off, nc, soff, q);
  };
  if (!(graph && !stall)) {
    rc = launch(s);
    if (rc == KS_OK) {
      g_batch.last_state_buf = buf;
      g_batch.last_state_off = soff;
    }
    return rc;
  }
  cudaStream_t cs = g_batch.capture_stream();
  KS_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  rc = launch(cs);
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &gr);
  if (rc == KS_OK && e != cudaSuccess) rc = cuda_rc(e);
  cudaGraphExec_t exec = nullptr;
  if (rc == KS_OK && (e = cudaGraphInstantiate(&exec, gr, 0)) != cudaSuccess) rc = cuda_rc(e);
  if (gr) cudaGraphDestroy(gr);
  if (rc != KS_OK) {
    cudaGetLastError();
    cudaFree(buf);
    return rc;
  }
  g_batch.graphs[key] = BatchState::Graph{exec, buf, soff};
  g_batch.last_state_buf = buf;
  g_batch.last_state_off = soff;
  return g_batch.launch_ordered(exec, s);
}

}  // namespace

extern "C" {

int ks_batch_status(void *stream) {
  std::lock_guard<std::mutex> lk(g_batch.mu);
  if (!g_batch.last_state_buf) return KS_OK;
  return persist_status(g_batch.last_state_buf, g_batch.last_state_off, (cudaStream_t)stream);
}


const char *ks_strerror(int code) {
  switch (code) {
    case KS_OK: return "ok";
    case KS_EINVAL: return "invalid argument";
    case KS_EPRIME: return "invalid modulus (not prime, not 1 mod 2N, too large or repeated)";
    case KS_ENOMEM: return "device allocation failed";
    case KS_ECUDA: return "CUDA error";
    case KS_ETIMEOUT: return "device-side wait timed out";
    case KS_EALIGN: return "pointer not 16-byte aligned";
    default: return "unknown error";
  }
}

const char *ks_cuda_error_string(void) { return cudaGetErrorString(g_last_cuda); }

int ks_context_create(const ks_params *prm, ks_context **out) {
  if (!prm || !out || !prm->q || !prm->p) return KS_EINVAL;
  *out = nullptr;
  const int logn = (int)prm->log2n, L = (int)prm->L, dnum = (int)prm->dnum;
  if (logn < 1 || logn > 17 || dnum < 1 || L < 0 || L + 1 > 128) return KS_EINVAL;
  const int nq = L + 1;
  const int alpha = (nq + dnum - 1) / dnum;
  if ((int)prm->nq != nq || (int)prm->np != alpha) return KS_EINVAL;
  return create_context(dnum, logn, L, (const u64 *)prm->q, (const u64 *)prm->p, alpha, nullptr,
                        out);
}

int ks_context_at_level(const ks_context *top, int level, ks_context **out) {
  if (!top || !out) return KS_EINVAL;
  *out = nullptr;
  if (top->top_L >= 0) return KS_EINVAL;  // a view of a view: take the top context
  if (level < 0 || level > top->L) return KS_EINVAL;
  std::vector<u64> q(top->mods.begin(), top->mods.begin() + level + 1);
  std::vector<u64> p(top->mods.begin() + top->nq, top->mods.end());
  return create_context(top->dnum, top->logn, level, q.data(), p.data(), top->alpha, top, out);
}

void ks_context_destroy(ks_context *c) {
  if (!c) return;
  forget_graphs(c);
  drop_graph_cache(c);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->table_mem) cudaFree(c->table_mem);
  if (c->ws) cudaFree(c->ws);
  if (c->stage) cudaFree(c->stage);
  delete c;
}

int ks_context_info(const ks_context *c, ks_info *info) {
  if (!c || !info) return KS_EINVAL;
  info->N = c->N;
  info->alpha = c->alpha;
  info->beta = c->beta;
  info->QP = c->qp;
  info->nq = c->nq;
  info->np = c->np;
  info->evk_words = (size_t)c->beta * 2 * c->eqp * c->N;
  info->L = c->L;
  info->top_L = c->top_L < 0 ? c->L : c->top_L;
  info->in_words = (size_t)c->nq * c->N;
  info->out_words = (size_t)2 * c->nq * c->N;
  info->table_bytes = c->table_bytes;
  info->tuned_variant = c->tuned_variant;
  info->tuned_chunks = c->tuned_chunks;
  info->tuned_batch = c->tuned_batch;
  info->tuned_ms = c->tuned_ms;
  info->selected_variant = c->sel_variant;
  info->selected_chunks = c->sel_chunks;
  info->tc = c->tc_ap > 0 ? 1 : 0;
  return KS_OK;
}

int ks_workspace_size(const ks_context *c, int variant, int chunks, size_t *bytes) {
  if (!c || !bytes) return KS_EINVAL;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  *bytes = pl.total * 8;
  return KS_OK;
}

int ks_switch(ks_context *c, const uint64_t *d, const uint64_t *evk, uint64_t *out, int variant,
              int chunks, void *ws, size_t ws_bytes, void *stream) {
  if (!c || !d || !evk || !out) return KS_EINVAL;
  if (!aligned16(d) || !aligned16(evk) || !aligned16(out) || (ws && !aligned16(ws)))
    return KS_EALIGN;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  return with_workspace(c, ws, ws_bytes, pl.total * 8, [&](u64 *base) {
    JobSet js = {};
    js.n = 1;
    js.j[0].d = (const u64 *)d;
    js.j[0].evk = (const u64 *)evk;
    js.j[0].out = (u64 *)out;
    js.j[0].ws = base;
    const std::array<uintptr_t, 10> key = {
        0, (uintptr_t)plan_code(pl), (uintptr_t)pl.chunks, (uintptr_t)d, (uintptr_t)evk, 0,
        (uintptr_t)out, (uintptr_t)base, (uintptr_t)s, 0};
    if (!use_graphs(c)) return run_plan(c, pl, js, s);
    return cached_launch(c, key, s, [&](cudaStream_t q) { return run_plan(c, pl, js, q); });
  });
}

}  // extern "C"

namespace ks {

// ks_switch on a caller workspace with every kernel launched directly on `stream`: no
// graph cache (no capture, instantiation or stream creation) and no context arena.
int switch_launch_only(ks_context *c, const uint64_t *d, const uint64_t *evk, uint64_t *out,
                       int variant, int chunks, void *ws, size_t ws_bytes, void *stream) {
  if (!c || !d || !evk || !out || !ws) return KS_EINVAL;
  if (!aligned16(d) || !aligned16(evk) || !aligned16(out) || !aligned16(ws)) return KS_EALIGN;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  if (ws_bytes < pl.total * 8) return KS_EINVAL;
  JobSet js = {};
  js.n = 1;
  js.j[0].d = (const u64 *)d;
  js.j[0].evk = (const u64 *)evk;
  js.j[0].out = (u64 *)out;
  js.j[0].ws = (u64 *)ws;
  return run_plan(c, pl, js, (cudaStream_t)stream, false);
}

}  // namespace ks

namespace {

// ks_switch_host_async_ws: host-buffer KeySwitch on the caller's scratch (workspace,
// device input, device output), with the transfers on the copy engines: the input is
// copied in, the kernels run on device buffers, the result is copied out, all queued on
// s. With calls on several streams the copies of one overlap the kernels of another
// (GPU-side accesses to mapped host memory, as ks_switch_host_async does, would instead
// occupy the first and last kernels for the whole transfer).
int switch_host_ws(ks_context *c, const uint64_t *d_host, const uint64_t *evk, uint64_t *out_host,
                   int variant, int chunks, void *ws, size_t ws_bytes, cudaStream_t s) {
  if (!c || !d_host || !evk || !out_host || !ws) return KS_EINVAL;
  if (!aligned16(evk) || !aligned16(ws)) return KS_EALIGN;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  const size_t in_w = (size_t)c->nq * c->N;
  if (ws_bytes < (pl.total + 3 * in_w) * 8) return KS_EINVAL;
  // pinned host memory only: pageable copies would not be asynchronous
  if (!host_mapped(d_host) || !host_mapped(out_host)) return KS_EINVAL;
  u64 *din = (u64 *)ws + pl.total, *dout = din + in_w;
  KS_TRY(cudaMemcpyAsync(din, d_host, in_w * 8, cudaMemcpyHostToDevice, s));
  JobSet js = {};
  js.n = 1;
  js.j[0].ws = (u64 *)ws;
  js.j[0].d = din;
  js.j[0].evk = (const u64 *)evk;
  js.j[0].out = dout;
  rc = run_plan(c, pl, js, s);
  if (rc) return rc;
  KS_TRY(cudaMemcpyAsync(out_host, dout, 2 * in_w * 8, cudaMemcpyDeviceToHost, s));
  return KS_OK;
}

// ks_switch_host / ks_switch_host_async. `async`: pinned buffers only, no final
// synchronization, and direct (chained) launches where ks_switch uses them.
int switch_host(ks_context *c, const uint64_t *d_host, const uint64_t *evk, uint64_t *out_host,
                int variant, int chunks, cudaStream_t s, bool async) {
  if (!c || !d_host || !evk || !out_host) return KS_EINVAL;
  const size_t in_b = (size_t)c->nq * c->N * 8, out_b = 2 * in_b;
  {
    std::lock_guard<std::mutex> lk(c->ws_mu);
    if (c->stage_bytes < in_b + out_b) {
      if (c->stage) {
        cudaDeviceSynchronize();
        cudaFree(c->stage);
      }
      c->stage = nullptr;
      c->stage_bytes = 0;
      if (cudaMalloc(&c->stage, in_b + out_b) != cudaSuccess) {
        cudaGetLastError();
        return KS_ENOMEM;
      }
      c->stage_bytes = in_b + out_b;
    }
  }
  uint64_t *din = (uint64_t *)c->stage;
  uint64_t *dout = din + (size_t)c->nq * c->N;
  if (!aligned16(evk)) return KS_EALIGN;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  // Pinned (device-mapped) host buffers: the first kernel reads the input from host
  // memory over the CPU-GPU link (leaving a device copy for the key multiply) and the
  // last kernel writes the result straight into host memory - no staging copies.
  // Otherwise: copy in, KeySwitch, copy out. Either way one cached graph per
  // (plan, buffers, stream) where it can be captured.
  const u64 *d_map = host_mapped(d_host);
  u64 *out_map = const_cast<u64 *>(host_mapped(out_host));
  const bool mapped = d_map && out_map;
  if (async && !mapped) return KS_EINVAL;
  // the kernels access mapped host buffers with 16-byte vector loads and stores
  if (mapped && (!aligned16(d_map) || !aligned16(out_map))) return KS_EALIGN;
  rc = with_workspace(c, nullptr, 0, pl.total * 8, [&](u64 *base) {
    JobSet js = {};
    js.n = 1;
    js.j[0].d = (const u64 *)din;
    js.j[0].evk = (const u64 *)evk;
    js.j[0].out = mapped ? out_map : (u64 *)dout;
    js.j[0].ws = base;
    js.j[0].dsrc = mapped ? d_map : nullptr;
    const std::array<uintptr_t, 10> key = {
        3, (uintptr_t)plan_code(pl), (uintptr_t)pl.chunks, (uintptr_t)d_host, (uintptr_t)evk,
        (uintptr_t)din, (uintptr_t)out_host, (uintptr_t)base, (uintptr_t)s, 0};
    if (async && !use_graphs(c)) return run_plan(c, pl, js, s);
    return cached_launch(c, key, s, [&](cudaStream_t q) {
      if (!mapped) KS_TRY(cudaMemcpyAsync(din, d_host, in_b, cudaMemcpyHostToDevice, q));
      const int r = run_plan(c, pl, js, q);
      if (r) return r;
      if (!mapped) KS_TRY(cudaMemcpyAsync(out_host, dout, out_b, cudaMemcpyDeviceToHost, q));
      return (int)KS_OK;
    });
  });
  if (rc || async) return rc;
  KS_TRY(cudaStreamSynchronize(s));
  return KS_OK;
}

}  // namespace

extern "C" {

int ks_switch_host(ks_context *c, const uint64_t *d_host, const uint64_t *evk, uint64_t *out_host,
                   int variant, int chunks, void *stream) {
  return switch_host(c, d_host, evk, out_host, variant, chunks, (cudaStream_t)stream, false);
}

int ks_switch_host_async(ks_context *c, const uint64_t *d_host, const uint64_t *evk,
                         uint64_t *out_host, int variant, int chunks, void *stream) {
  return switch_host(c, d_host, evk, out_host, variant, chunks, (cudaStream_t)stream, true);
}

int ks_host_workspace_size(const ks_context *c, int variant, int chunks, size_t *bytes) {
  if (!c || !bytes) return KS_EINVAL;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  *bytes = (pl.total + 3 * (size_t)c->nq * c->N) * 8;
  return KS_OK;
}

int ks_switch_host_async_ws(ks_context *c, const uint64_t *d_host, const uint64_t *evk,
                            uint64_t *out_host, int variant, int chunks, void *ws,
                            size_t ws_bytes, void *stream) {
  return switch_host_ws(c, d_host, evk, out_host, variant, chunks, ws, ws_bytes,
                        (cudaStream_t)stream);
}

int ks_keygen(ks_context *c, const int8_t *s_from, const int8_t *s_to, const uint64_t *a,
              const int32_t *e, uint64_t *evk, void *stream) {
  return keygen_impl(c, s_from, s_to, 0, false, a, e, evk, stream);
}

int ks_keygen_relin(ks_context *c, const int8_t *s, const uint64_t *a, const int32_t *e,
                    uint64_t *evk, void *stream) {
  return keygen_impl(c, s, s, 0, true, a, e, evk, stream);
}

int ks_keygen_galois(ks_context *c, const int8_t *s, uint32_t galois_elt, const uint64_t *a,
                     const int32_t *e, uint64_t *evk, void *stream) {
  if (!c || !galois_ok(c, galois_elt)) return KS_EINVAL;
  const u64 two_n = (u64)2 * c->N;
  // k^-1 mod 2N by Newton iteration (k odd): x <- x (2 - k x) doubles the correct bits
  u64 inv = galois_elt;
  for (int it = 0; it < 5; ++it) inv = (inv * (2 - (u64)galois_elt * inv)) & (two_n - 1);
  return keygen_impl(c, s, s, (unsigned)inv, false, a, e, evk, stream);
}

int ks_eval_workspace_size(const ks_context *c, int op, int variant, int chunks, size_t *bytes) {
  if (!c || !bytes || op < KS_OP_SWITCH || op > KS_OP_HROT) return KS_EINVAL;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  *bytes = (pl.total + (size_t)op * c->nq * c->N) * 8;
  return KS_OK;
}

int ks_hmul(ks_context *c, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *rlk,
            uint64_t *out, int variant, int chunks, void *ws, size_t ws_bytes, void *stream) {
  if (!c || !ct1 || !ct2 || !rlk || !out) return KS_EINVAL;
  if (!aligned16(ct1) || !aligned16(ct2) || !aligned16(rlk) || !aligned16(out) ||
      (ws && !aligned16(ws)))
    return KS_EALIGN;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  const size_t extra = (size_t)c->nq * c->N;
  cudaStream_t s = (cudaStream_t)stream;
  return with_workspace(c, ws, ws_bytes, (pl.total + extra) * 8, [&](u64 *base) {
    u64 *d2 = base + pl.total;
    JobSet js = {};
    js.n = 1;
    js.j[0].d = d2;
    js.j[0].evk = (const u64 *)rlk;
    js.j[0].out = (u64 *)out;
    js.j[0].ws = base;
    js.j[0].add = (const u64 *)out;
    js.j[0].addmask = 3;
    const std::array<uintptr_t, 10> key = {
        1, (uintptr_t)plan_code(pl), (uintptr_t)pl.chunks, (uintptr_t)ct1, (uintptr_t)ct2,
        (uintptr_t)rlk, (uintptr_t)out, (uintptr_t)base, (uintptr_t)s, 0};
    auto enqueue = [&](cudaStream_t q) {
      KS_TRY(launch_tensor(c, (const u64 *)ct1, (const u64 *)ct2, (u64 *)out, d2, q));
      return run_plan(c, pl, js, q);
    };
    return use_graphs(c) ? cached_launch(c, key, s, enqueue) : enqueue(s);
  });
}

int ks_hrot(ks_context *c, const uint64_t *ct, uint32_t galois_elt, const uint64_t *rtk,
            uint64_t *out, int variant, int chunks, void *ws, size_t ws_bytes, void *stream) {
  if (!c || !ct || !rtk || !out || !galois_ok(c, galois_elt)) return KS_EINVAL;
  if (!aligned16(ct) || !aligned16(rtk) || !aligned16(out) || (ws && !aligned16(ws)))
    return KS_EALIGN;
  Plan pl;
  int rc = make_plan(c, variant, chunks, &pl);
  if (rc) return rc;
  const size_t extra = (size_t)2 * c->nq * c->N;
  cudaStream_t s = (cudaStream_t)stream;
  return with_workspace(c, ws, ws_bytes, (pl.total + extra) * 8, [&](u64 *base) {
    u64 *y0 = base + pl.total, *y1 = y0 + (size_t)c->nq * c->N;
    JobSet js = {};
    js.n = 1;
    js.j[0].d = y1;
    js.j[0].evk = (const u64 *)rtk;
    js.j[0].out = (u64 *)out;
    js.j[0].ws = base;
    js.j[0].add = y0;  // out_0 += sigma(ct_0); out_1 is the KeySwitch's alone
    js.j[0].addmask = 1;
    const std::array<uintptr_t, 10> key = {
        2, (uintptr_t)plan_code(pl), (uintptr_t)pl.chunks, (uintptr_t)ct, (uintptr_t)galois_elt,
        (uintptr_t)rtk, (uintptr_t)out, (uintptr_t)base, (uintptr_t)s, 0};
    auto enqueue = [&](cudaStream_t q) {
      KS_TRY(launch_automorph(c, (const u64 *)ct, galois_elt, y0, y1, q));
      return run_plan(c, pl, js, q);
    };
    return use_graphs(c) ? cached_launch(c, key, s, enqueue) : enqueue(s);
  });
}

int ks_switch_batch(const ks_job *jobs, int njobs, int flags, void *stream) {
  if (njobs < 0 || (njobs > 0 && !jobs)) return KS_EINVAL;
  if (flags & ~(KS_BATCH_GRAPH | KS_BATCH_AUTOTUNE | KS_BATCH_PERSISTENT | KS_BATCH_SELECT |
                KS_BATCH_TEST_STALL))
    return KS_EINVAL;
  if ((flags & KS_BATCH_SELECT) && (flags & (KS_BATCH_AUTOTUNE | KS_BATCH_PERSISTENT)))
    return KS_EINVAL;
  if (njobs == 0) return KS_OK;
  for (int k = 0; k < njobs; ++k) {
    const ks_job &jb = jobs[k];
    if (!jb.ctx || !jb.d_dev || !jb.evk_dev || !jb.out_dev) return KS_EINVAL;
    if (!aligned16(jb.d_dev) || !aligned16(jb.evk_dev) || !aligned16(jb.out_dev))
      return KS_EALIGN;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (flags & KS_BATCH_PERSISTENT) return batch_persistent(jobs, njobs, flags, s);
  if (flags & KS_BATCH_TEST_STALL) return KS_EINVAL;
  // Groups of jobs sharing a context and a plan, in order of first appearance.
  std::vector<ks_context *> ctxs;
  std::vector<std::pair<int, int>> gplan;  // requested (variant, chunks)
  std::vector<std::vector<int>> members;
  for (int k = 0; k < njobs; ++k) {
    size_t g = 0;
    while (g < ctxs.size() && !(ctxs[g] == jobs[k].ctx && gplan[g].first == jobs[k].variant &&
                                gplan[g].second == jobs[k].chunks))
      ++g;
    if (g == ctxs.size()) {
      ctxs.push_back(jobs[k].ctx);
      gplan.emplace_back(jobs[k].variant, jobs[k].chunks);
      members.emplace_back();
    }
    members[g].push_back(k);
  }
  if (flags & KS_BATCH_AUTOTUNE) {
    for (size_t g = 0; g < ctxs.size(); ++g) {
      ks_context *c = ctxs[g];
      if ((gplan[g].first & 0xff) != KS_AUTO) continue;  // the job names its plan
      if (c->tuned_batch == std::min<int>(kMaxBatch, (int)members[g].size()) &&
          c->tuned_variant > 0)
        continue;
      const ks_job &jb = jobs[members[g][0]];
      int v = 0, ch = 0;
      int rc = ks_tune(c, jb.d_dev, jb.evk_dev, jb.out_dev,
                       std::min<int>(kMaxBatch, (int)members[g].size()), &v, &ch, stream);
      if (rc) return rc;
    }
  }
  if (flags & KS_BATCH_SELECT) {
    for (size_t g = 0; g < ctxs.size(); ++g) {
      ks_context *c = ctxs[g];
      if ((gplan[g].first & 0xff) != KS_AUTO) continue;  // the job names its plan
      if (!selected_current(c)) {
        int rc = ks_select(c, nullptr, nullptr, stream);
        if (rc) return rc;
      }
      gplan[g] = {selected_plan(c) | (gplan[g].first & ~0xff),
                  gplan[g].second ? gplan[g].second : c->sel_chunks};
    }
  }
  std::vector<Plan> plans(ctxs.size());
  size_t total = 0;
  for (size_t g = 0; g < ctxs.size(); ++g) {
    int rc = make_plan(ctxs[g], gplan[g].first, gplan[g].second, &plans[g]);
    if (rc) return rc;
    total += plans[g].total * 8 * members[g].size();
  }
  std::lock_guard<std::mutex> lk(g_batch.mu);
  if (g_batch.arena_bytes < total) {
    if (g_batch.arena) {
      cudaDeviceSynchronize();
      cudaFree(g_batch.arena);
    }
    clear_graphs_locked();
    g_batch.arena = nullptr;
    g_batch.arena_bytes = 0;
    if (cudaMalloc(&g_batch.arena, total) != cudaSuccess) {
      cudaGetLastError();
      return KS_ENOMEM;
    }
    g_batch.arena_bytes = total;
  }
  std::vector<uintptr_t> key;
  const bool graph = (flags & KS_BATCH_GRAPH) != 0;
  if (graph) {
    key.push_back((uintptr_t)njobs);
    key.push_back((uintptr_t)s);
    for (int k = 0; k < njobs; ++k) {
      key.push_back((uintptr_t)jobs[k].ctx);
      key.push_back((uintptr_t)jobs[k].d_dev);
      key.push_back((uintptr_t)jobs[k].evk_dev);
      key.push_back((uintptr_t)jobs[k].out_dev);
      key.push_back(((uintptr_t)(uint32_t)jobs[k].variant << 32) | (uint32_t)jobs[k].chunks);
    }
    // every input of a group's plan: its (selected) request and the context's choices
    for (size_t g = 0; g < ctxs.size(); ++g) {
      key.push_back(((uintptr_t)(uint32_t)gplan[g].first << 32) | (uint32_t)gplan[g].second);
      key.push_back(((uintptr_t)(uint32_t)ctxs[g]->tuned_variant << 32) |
                    (uint32_t)ctxs[g]->tuned_chunks);
      key.push_back(((uintptr_t)(uint32_t)ctxs[g]->sel_variant << 32) |
                    (uint32_t)ctxs[g]->sel_chunks);
    }
    auto it = g_batch.graphs.find(key);
    if (it != g_batch.graphs.end()) return g_batch.launch_ordered(it->second.exec, s);
  }
  // A graph is captured on an internal stream (the caller's may be the legacy default
  // stream, which cannot be captured) and launched ordered after `s`.
  const cudaStream_t caller = s;
  if (graph) {
    s = g_batch.capture_stream();
    KS_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  }
  const bool prof = g_prof.on;
  if (graph) g_prof.on = false;
  // Enqueue: each context group on its own stream (fork from s, join back to s);
  // inside a group, up to kMaxBatch jobs share each launch (grid z).
  int rc = KS_OK;
  {
    const int G = (int)ctxs.size();
    cudaEvent_t fork = nullptr;
    if (G > 1) {
      fork = g_batch.event();
      cudaEventRecord(fork, s);
    }
    // Largest groups first, each on the internal stream with the least work so far
    // (longest-processing-time order): the big jobs of an uneven batch start at once,
    // on different streams, and the small ones fill in behind them. Work ~ the
    // NTT volume beta * QP * N log N of a job.
    std::vector<int> order(G), sid(G, 0);
    std::vector<double> cost(G);
    for (int g = 0; g < G; ++g) {
      order[g] = g;
      const ks_context *c = ctxs[g];
      cost[g] = (double)members[g].size() * c->beta * c->qp * c->N * c->logn;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    {
      double load[kBatchStreams] = {};
      for (int g : order) {
        int k = 0;
        for (int q = 1; q < kBatchStreams; ++q)
          if (load[q] < load[k]) k = q;
        sid[g] = k;
        load[k] += cost[g];
      }
    }
    char *base = (char *)g_batch.arena;
    for (int oi = 0; oi < G && rc == KS_OK; ++oi) {
      const int g = order[oi];
      cudaStream_t sg = s;
      if (G > 1) {
        sg = g_batch.stream(sid[g]);
        cudaStreamWaitEvent(sg, fork, 0);
      }
      const Plan &pl = plans[g];
      const std::vector<int> &mem = members[g];
      for (size_t k0 = 0; k0 < mem.size() && rc == KS_OK; k0 += kMaxBatch) {
        JobSet js = {};
        js.n = (int)std::min<size_t>(kMaxBatch, mem.size() - k0);
        for (int q = 0; q < js.n; ++q) {
          const ks_job &jb = jobs[mem[k0 + q]];
          js.j[q].d = (const u64 *)jb.d_dev;
          js.j[q].evk = (const u64 *)jb.evk_dev;
          js.j[q].out = (u64 *)jb.out_dev;
          js.j[q].ws = (u64 *)base;
          base += pl.total * 8;
        }
        rc = run_plan(ctxs[g], pl, js, sg);
      }
      if (G > 1) {
        cudaEvent_t done = g_batch.event();
        cudaEventRecord(done, sg);
        cudaStreamWaitEvent(s, done, 0);
      }
    }
  }
  g_prof.on = prof;
  if (graph) {
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &gr);
    if (rc == KS_OK && e != cudaSuccess) rc = cuda_rc(e);
    cudaGraphExec_t exec = nullptr;
    if (rc == KS_OK) {
      e = cudaGraphInstantiate(&exec, gr, 0);
      if (e != cudaSuccess) rc = cuda_rc(e);
    }
    if (gr) cudaGraphDestroy(gr);
    if (rc != KS_OK) {
      cudaGetLastError();
      return rc;
    }
    g_batch.graphs[key] = BatchState::Graph{exec, nullptr, 0};
    return g_batch.launch_ordered(exec, caller);
  }
  return rc;
}

int ks_tune(ks_context *c, const uint64_t *d, const uint64_t *evk, uint64_t *out, int batch,
            int *variant, int *chunks, void *stream) {
  if (!c || !d || !evk || !out || batch < 1 || batch > kMaxBatch) return KS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int bases[][2] = {{KS_DPOB, 0}, {KS_DSOB, 0}, {KS_DPOC, 2}, {KS_DPOC, 4}, {KS_DSOC, 2}};
  size_t ws_max = 0;
  const int radix[3] = {0, KS_RADIX4, KS_RADIX16};
  for (auto &b : bases)
    for (int r : radix) {
      Plan pl;
      if (make_plan(c, b[0] | r | KS_BCONV_TC, b[1], &pl) == KS_OK)
        ws_max = std::max(ws_max, pl.total * 8);
    }
  const size_t out_b = (size_t)2 * c->nq * c->N * 8;
  void *mem = nullptr;
  if (cudaMalloc(&mem, batch * (ws_max + out_b)) != cudaSuccess) {
    cudaGetLastError();
    return KS_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool prof = g_prof.on;
  g_prof.on = false;
  int rc = KS_OK;
  // best of `reps` timed launch sets (after one untimed) of plan (v, ch), ms
  auto time_plan = [&](int v, int ch, int reps) -> float {
    Plan pl;
    if (make_plan(c, v, ch, &pl) != KS_OK) return 1e30f;
    JobSet js = {};
    js.n = batch;
    for (int q = 0; q < batch; ++q) {
      char *base = (char *)mem + q * (ws_max + out_b);
      js.j[q].d = (const u64 *)d;
      js.j[q].evk = (const u64 *)evk;
      js.j[q].out = (u64 *)(base + ws_max);
      js.j[q].ws = (u64 *)base;
    }
    float ms_min = 1e30f;
    for (int rep = 0; rep <= reps && rc == KS_OK; ++rep) {
      cudaEventRecord(e0, s);
      rc = run_plan(c, pl, js, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = KS_ECUDA;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) ms_min = std::min(ms_min, ms);
    }
    return ms_min;
  };
  // 1) dataflow x radix
  float best = 1e30f;
  int best_v = KS_DPOB, best_c = 0;
  for (auto &b : bases)
    for (int ri = 0; ri < 3 && rc == KS_OK; ++ri) {
      const int v = b[0] | radix[ri];
      const float ms = time_plan(v, b[1], 3);
      if (ms < best) {
        best = ms;
        best_v = v;
        best_c = b[1];
      }
    }
  // 2) the schedule of the winner, one coordinate at a time: each stage's radix, then the
  // tensor-core basis conversions (both, else the ModDown one alone; a column pass they
  // replace drops its radix), then each remaining column pass's tile, then the split
  // ModDown. The winner is re-timed with the same number of repetitions, and a change is
  // kept only if the whole KeySwitch gets faster by more than the timing noise (1.5%).
  if (rc == KS_OK && c->loga > 0) {
    best = time_plan(best_v, best_c, 6);
    const int plan_code3 = (best_v & KS_RADIX4) ? KS_R4 : (best_v & KS_RADIX16) ? KS_R16 : KS_R8;
    for (int st = 0; st < ST_COUNT && rc == KS_OK; ++st)
      for (int code = KS_R4; code <= KS_R16 && rc == KS_OK; ++code) {
        if (code == plan_code3) continue;
        const int cur = (best_v >> (KS_STAGE_SHIFT + 2 * st)) & 3;
        if (cur == code) continue;
        const int v = (best_v & ~KS_STAGE_RADIX(st, 3)) | KS_STAGE_RADIX(st, code);
        const float ms = time_plan(v, best_c, 6);
        if (ms < 0.985f * best) {
          best = ms;
          best_v = v;
        }
      }
    if (rc == KS_OK && c->tc_ap > 0 && !(best_v & KS_UNFUSED)) {
      const int up_dn = KS_STAGE_RADIX(ST_UPC, 3) | KS_STAGE_RADIX(ST_DNC, 3);
      const int cand[2] = {(best_v & ~up_dn) | KS_BCONV_TC,
                           (best_v & ~KS_STAGE_RADIX(ST_DNC, 3)) | KS_BCONV_TC_DOWN};
      for (int v : cand) {
        if (rc != KS_OK) break;
        const float ms = time_plan(v, best_c, 6);
        if (ms < 0.985f * best) {
          best = ms;
          best_v = v;
          break;
        }
      }
    }
    const bool tc_up = (best_v & KS_BCONV_TC) != 0;
    const bool tc_down = (best_v & (KS_BCONV_TC | KS_BCONV_TC_DOWN)) != 0;
    for (int bit : {KS_COLALT_INV, KS_COLALT_UPC, KS_COLALT_DNC, KS_SPLIT_DOWN}) {
      if (rc != KS_OK) break;
      if ((tc_up && bit == KS_COLALT_UPC) || (tc_down && bit == KS_COLALT_DNC)) continue;
      if (bit == KS_SPLIT_DOWN && ((best_v & 0xff) != KS_DPOB || (best_v & KS_UNFUSED))) continue;
      const float ms = time_plan(best_v ^ bit, best_c, 6);
      if (ms < 0.985f * best) {
        best = ms;
        best_v ^= bit;
      }
    }
  }
  g_prof.on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == KS_OK) {
    // leave the caller's out with the switched result (every candidate computes it)
    Plan pl;
    make_plan(c, best_v, best_c, &pl);
    JobSet js = {};
    js.n = 1;
    js.j[0].d = (const u64 *)d;
    js.j[0].evk = (const u64 *)evk;
    js.j[0].out = (u64 *)out;
    js.j[0].ws = (u64 *)mem;
    rc = run_plan(c, pl, js, s);
    if (rc == KS_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = KS_ECUDA;
  }
  cudaFree(mem);
  if (rc) return rc;
  c->tuned_variant = best_v;
  c->tuned_chunks = best_c;
  c->tuned_batch = batch;
  c->tuned_ms = best / batch;
  if (variant) *variant = best_v;
  if (chunks) *chunks = best_c;
  return KS_OK;
}

int ks_profile_begin(void) {
  g_prof.on = true;
  return KS_OK;
}

int ks_profile_end(ks_kernel_stat *stats, int max_stats, int *count) {
  g_prof.on = false;
  std::vector<ks_kernel_stat> agg;
  int rc = KS_OK;
  for (auto &r : g_prof.recs) {
    float ms = 0;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) rc = cuda_rc(e);
    ks_kernel_stat *hit = nullptr;
    for (auto &x : agg)
      if (std::strncmp(x.name, r.name, sizeof(x.name)) == 0) hit = &x;
    if (!hit) {
      agg.push_back(ks_kernel_stat{});
      hit = &agg.back();
      std::strncpy(hit->name, r.name, sizeof(hit->name) - 1);
    }
    hit->launches += 1;
    hit->ms += ms;
    hit->bytes += r.bytes;
    hit->ops += r.ops;
    hit->macs += r.macs;
    hit->tensor_flops += r.tflops;
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
  if (count) *count = (int)agg.size();
  if (stats)
    for (int k = 0; k < (int)agg.size() && k < max_stats; ++k) stats[k] = agg[k];
  return rc;
}

int ks_sync_status(ks_context *c, void *stream) {
  if (!c) return KS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  KS_TRY(cudaMemcpyAsync(&h, c->tab.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  KS_TRY(cudaStreamSynchronize(s));
  if (h) {
    KS_TRY(cudaMemsetAsync(c->tab.err, 0, sizeof(int), s));
    KS_TRY(cudaStreamSynchronize(s));
    return KS_ETIMEOUT;
  }
  return KS_OK;
}

}  // extern "C"
