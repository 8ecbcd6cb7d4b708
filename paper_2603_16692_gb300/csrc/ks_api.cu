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
#include <new>

#include "ks_internal.h"
#include "ks_ntt.cuh"

using namespace ks;

namespace {

struct Plan {
  int base;      // KS_DSOB..KS_DPOC
  bool unfused;
  int chunks;    // phase-1 and phase-2 group counts (1 for OB)
  int clen;      // max QP-limbs per phase-1 group
  int clq;       // max Q-limbs per phase-2 group
  size_t off_v, off_tmp, off_acc, off_vp, off_tmp2, total;  // in u64 words
  size_t tmp_slots, tmp2_slots;
};

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

int make_plan(const ks_context *c, int variant, int chunks, Plan *pl) {
  int base = variant & 0xff;
  if (variant & ~(0xff | KS_UNFUSED)) return KS_EINVAL;
  if (base == KS_AUTO) base = KS_DPOB;
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
  double bytes, ops;
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

// Run one launcher; when profiling, bracket it with events on its stream.
template <class F>
cudaError_t timed(const char *name, double bytes, double ops, cudaStream_t s, F f) {
  if (!g_prof.on) return f();
  cudaEvent_t a = g_prof.get(), b = g_prof.get();
  cudaEventRecord(a, s);
  cudaError_t e = f();
  cudaEventRecord(b, s);
  g_prof.recs.push_back({name, a, b, bytes, ops});
  return e;
}

int run_plan(ks_context *c, const Plan &pl, const u64 *d, const u64 *evk, u64 *out, u64 *ws,
             cudaStream_t s) {
  const size_t N = c->N;
  const double W = (double)N * 8;                       // bytes per limb
  const double BF_A = (double)N / 2 * c->loga;          // butterflies, column pass
  const double BF_B = (double)N / 2 * c->logb;          // butterflies, row pass
  const bool single = c->loga == 0;
  const LaunchTable &L = *c->lt;
  u64 *v = ws + pl.off_v, *tmp = ws + pl.off_tmp, *acc = ws + pl.off_acc, *vp = ws + pl.off_vp,
      *tmp2 = ws + pl.off_tmp2;
  const bool dp = pl.base == KS_DPOB || pl.base == KS_DPOC;
  const bool oc = pl.base == KS_DSOC || pl.base == KS_DPOC;
  static thread_local TaskList tl, tg;
  static thread_local std::vector<uint32_t> big;
  auto dsize = [&](int j) { return std::min(c->nq, (j + 1) * c->alpha) - j * c->alpha; };

  // Input iNTT, fused with the per-limb factor N^-1 * Qhat_{j,i}^-1 of the ModUp BConv.
  {
    const double nl = c->nq;
    KS_TRY(timed("intt_row(d)", 2 * nl * W, nl * (BF_B + (single ? N : 0)), s, [&] {
      return L.intt_row(c, d, 0, v, 0, 1, c->nq, 0, c->tab.iscale_q, s);
    }));
    if (!single)
      KS_TRY(timed("intt_col(d)", 2 * nl * W, nl * (BF_A + N), s, [&] {
        return L.intt_col(c, v, 0, 1, c->nq, 0, c->tab.iscale_q, s);
      }));
  }

  // Phase 1: ModUp (BConv + NTT) and key multiply, per output group.
  for (int ch = 0; ch < pl.chunks; ++ch) {
    const int t0 = ch * pl.clen, t1 = std::min(c->qp, t0 + pl.clen);
    if (t0 >= t1) continue;
    tg.n = 0;
    for (int t = t0; t < t1; ++t) tg.t[tg.n++] = pack_task(t, 0, 0);
    SlotMap sm;
    sm.st = 1;
    sm.base = oc ? -t0 : 0;
    sm.sj = dp ? (oc ? pl.clen : c->qp) : 0;
    const int jstep = dp ? c->beta : 1;
    for (int j0 = 0; j0 < c->beta; j0 += jstep) {
      const int j1 = j0 + jstep;
      big.clear();
      double src_b = 0, conv_ops = 0, own = 0;
      for (int j = j0; j < j1; ++j) {
        const int lo = j * c->alpha, hi = lo + dsize(j);
        src_b += dsize(j) * W;
        for (int t = t0; t < t1; ++t) {
          if (t >= lo && t < hi) {
            own += 1;
            continue;
          }
          big.push_back(pack_task(t, j, j * sm.sj + t * sm.st + sm.base));
          conv_ops += (double)N * (dsize(j) + 1);
        }
      }
      const double nconv = (double)big.size(), nt = tg.n, nd = j1 - j0;
      const bool first = j0 == 0;
      for (size_t p0 = 0; p0 < big.size(); p0 += kMaxTasks) {
        tl.n = (int)std::min<size_t>(kMaxTasks, big.size() - p0);
        std::memcpy(tl.t, big.data() + p0, tl.n * sizeof(uint32_t));
        const double f = (double)tl.n / std::max(1.0, nconv);
        if (!pl.unfused) {
          if (!single)
            KS_TRY(timed("modup_col", tl.n * W + f * src_b, f * conv_ops + tl.n * BF_A, s,
                         [&] { return L.modup_col(c, tl, v, tmp, s); }));
        } else {
          KS_TRY(timed("bconv_up", tl.n * W + f * src_b, f * conv_ops, s,
                       [&] { return launch_bconv_up(c, tl, v, tmp, s); }));
          if (!single)
            KS_TRY(timed("ntt_col", 2 * tl.n * W, tl.n * BF_A, s,
                         [&] { return L.ntt_col(c, tl, tmp, s); }));
          KS_TRY(timed("ntt_row", 2 * tl.n * W, tl.n * BF_B, s,
                       [&] { return L.ntt_row(c, tl, tmp, s); }));
        }
      }
      // key multiply: evk 2 words per (digit, target); ext from tmp (or d on own limbs);
      // acc written (and read when accumulating over digit launches)
      const double km_bytes = (2 * nd * nt + nconv + own + (first ? 2 : 4) * nt) * W;
      const double km_ops = 2 * nd * nt * N + own * N;
      if (!pl.unfused) {
        const double b = km_bytes + (single ? src_b - nconv * W : 0);
        const double o = km_ops + nconv * BF_B + (single ? conv_ops : 0);
        KS_TRY(timed("modup_row_keymult", b, o, s, [&] {
          return L.modup_row(c, tg, j0, j1, sm, first, d, v, tmp, evk, acc, s);
        }));
      } else {
        KS_TRY(timed("keymult", km_bytes, km_ops, s, [&] {
          return launch_keymult(c, tg, j0, j1, sm, first, d, tmp, evk, acc, s);
        }));
      }
    }
  }

  // iNTT of the P-limbs of both accumulators, fused with N^-1 * Phat_k^-1.
  {
    const double nl = 2.0 * c->np;
    KS_TRY(timed("intt_row(accP)", 2 * nl * W, nl * (BF_B + (single ? N : 0)), s, [&] {
      return L.intt_row(c, acc + (size_t)c->nq * N, c->qp, vp, c->np, 2, c->np, c->nq,
                        c->tab.iscale_p, s);
    }));
    if (!single)
      KS_TRY(timed("intt_col(accP)", 2 * nl * W, nl * (BF_A + N), s, [&] {
        return L.intt_col(c, vp, c->np, 2, c->np, c->nq, c->tab.iscale_p, s);
      }));
  }

  // Phase 2: ModDown (BConv P->Q + NTT) and (acc - .) * P^-1, per output group.
  for (int ch = 0; ch < pl.chunks; ++ch) {
    const int i0 = ch * pl.clq, i1 = std::min(c->nq, i0 + pl.clq);
    if (i0 >= i1) continue;
    const int span = oc ? pl.clq : c->nq;
    const int ibase = oc ? i0 : 0;
    tl.n = 0;
    for (int cc = 0; cc < 2; ++cc)
      for (int i = i0; i < i1; ++i) tl.t[tl.n++] = pack_task(i, cc, cc * span + (i - ibase));
    tg.n = 0;
    for (int i = i0; i < i1; ++i) tg.t[tg.n++] = pack_task(i, 0, i - ibase);
    const double n = tl.n, vp_b = 2.0 * c->np * W, conv = n * N * (c->np + 1.0);
    if (!pl.unfused) {
      if (!single)
        KS_TRY(timed("moddown_col", n * W + vp_b, conv + n * BF_A, s,
                     [&] { return L.moddown_col(c, tl, vp, tmp2, s); }));
      const double b = 3 * n * W + (single ? vp_b - n * W : 0);
      const double o = n * (BF_B + N) + (single ? conv : 0);
      KS_TRY(timed("moddown_row", b, o, s, [&] {
        return L.moddown_row(c, tg, span, vp, tmp2, acc, out, s);
      }));
    } else {
      KS_TRY(timed("bconv_down", n * W + vp_b, conv, s,
                   [&] { return launch_bconv_down(c, tl, vp, tmp2, s); }));
      if (!single)
        KS_TRY(timed("ntt_col", 2 * n * W, n * BF_A, s,
                     [&] { return L.ntt_col(c, tl, tmp2, s); }));
      KS_TRY(timed("ntt_row", 2 * n * W, n * BF_B, s, [&] { return L.ntt_row(c, tl, tmp2, s); }));
      KS_TRY(timed("moddown_scale", 3 * n * W, n * N, s,
                   [&] { return launch_moddown_scale(c, tl, tmp2, acc, out, s); }));
    }
  }
  return KS_OK;
}

}  // namespace

extern "C" {

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
  const int beta = (nq + alpha - 1) / alpha;
  if ((int)prm->nq != nq || (int)prm->np != alpha) return KS_EINVAL;
  const int qp = nq + alpha;
  if (qp > kMaxLimbs) return KS_EINVAL;
  std::vector<u64> mods(prm->q, prm->q + nq);
  mods.insert(mods.end(), prm->p, prm->p + alpha);
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
  c->N = 1 << logn;
  c->loga = ks::geo_loga(logn);
  c->logb = logn - c->loga;
  c->loggr = ks::geo_loggr(logn);
  c->lt = ks::launch_table(logn);
  if (!c->lt) {
    delete c;
    return KS_EINVAL;
  }
  c->mods = mods;
  // basis-conversion sums: run * max_source * m < m 2^64
  c->run_up = (int)std::min<u64>(1 << 20, (~(u64)0) / maxq);
  c->run_down = (int)std::min<u64>(1 << 20, (~(u64)0) / maxp);
  cudaGetDevice(&c->device);
  int rc = ks::build_tables(c);
  if (rc) {
    delete c;
    return rc;
  }
  *out = c;
  return KS_OK;
}

void ks_context_destroy(ks_context *c) {
  if (!c) return;
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
  info->evk_words = (size_t)c->beta * 2 * c->qp * c->N;
  info->in_words = (size_t)c->nq * c->N;
  info->out_words = (size_t)2 * c->nq * c->N;
  info->table_bytes = c->table_bytes;
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
  const size_t need = pl.total * 8;
  cudaStream_t s = (cudaStream_t)stream;
  if (ws) {
    if (ws_bytes < need) return KS_EINVAL;
    return run_plan(c, pl, (const u64 *)d, (const u64 *)evk, (u64 *)out, (u64 *)ws, s);
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
  return run_plan(c, pl, (const u64 *)d, (const u64 *)evk, (u64 *)out, (u64 *)c->ws, s);
}

int ks_switch_host(ks_context *c, const uint64_t *d_host, const uint64_t *evk, uint64_t *out_host,
                   int variant, int chunks, void *stream) {
  if (!c || !d_host || !evk || !out_host) return KS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
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
  KS_TRY(cudaMemcpyAsync(din, d_host, in_b, cudaMemcpyHostToDevice, s));
  int rc = ks_switch(c, din, evk, dout, variant, chunks, nullptr, 0, stream);
  if (rc) return rc;
  KS_TRY(cudaMemcpyAsync(out_host, dout, out_b, cudaMemcpyDeviceToHost, s));
  KS_TRY(cudaStreamSynchronize(s));
  return KS_OK;
}

int ks_keygen(ks_context *c, const int8_t *s_from, const int8_t *s_to, const uint64_t *a,
              const int32_t *e, uint64_t *evk, void *stream) {
  if (!c || !s_from || !s_to || !a || !e || !evk) return KS_EINVAL;
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
    cudaError_t err = launch_keygen_lift(c, s_from, s_to, e, polys, s);
    if (err) { rc = cuda_rc(err); break; }
    // transform every lifted limb in place (task lists of at most kMaxTasks)
    for (int k0 = 0; k0 < npoly * c->qp; k0 += kMaxTasks) {
      TaskList part;
      part.n = std::min(kMaxTasks, npoly * c->qp - k0);
      for (int k = 0; k < part.n; ++k) part.t[k] = pack_task((k0 + k) % c->qp, 0, k0 + k);
      err = c->lt->ntt_col(c, part, polys, s);
      if (!err) err = c->lt->ntt_row(c, part, polys, s);
      if (err) break;
    }
    if (err) { rc = cuda_rc(err); break; }
    err = launch_keygen_combine(c, polys, (const u64 *)a, (u64 *)evk, s);
    if (err) { rc = cuda_rc(err); break; }
    err = cudaStreamSynchronize(s);
    if (err) rc = cuda_rc(err);
  } while (0);
  cudaFree(polys);
  return rc;
}

int ks_switch_batch(const ks_job *jobs, int njobs, int flags, void *stream) {
  if (njobs < 0 || (njobs > 0 && !jobs)) return KS_EINVAL;
  (void)flags;
  for (int k = 0; k < njobs; ++k) {
    int rc = ks_switch(jobs[k].ctx, jobs[k].d_dev, jobs[k].evk_dev, jobs[k].out_dev, KS_AUTO, 0,
                       nullptr, 0, stream);
    if (rc) return rc;
  }
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
