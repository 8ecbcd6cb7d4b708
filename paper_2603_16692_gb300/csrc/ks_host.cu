// Host-side set-up of a KeySwitch context: parameter checks and the constant
// tables (twiddles in the two-pass layouts, basis-conversion constants with
// their Montgomery factors, iNTT scales, P^-1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "ks_internal.h"
#include "ks_ntt.cuh"

namespace ks {

namespace {

typedef unsigned __int128 u128;

u64 mulm(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }

u64 powm(u64 b, u64 e, u64 m) {
  u64 r = 1 % m;
  b %= m;
  for (; e; e >>= 1) {
    if (e & 1) r = mulm(r, b, m);
    b = mulm(b, b, m);
  }
  return r;
}

// Inverse mod m by the extended Euclidean algorithm (m prime, a != 0 mod m).
u64 invm(u64 a, u64 m) {
  __int128 t = 0, nt = 1, r = m, nr = a % m;
  while (nr != 0) {
    __int128 q = r / nr;
    __int128 tmp = t - q * nt;
    t = nt;
    nt = tmp;
    tmp = r - q * nr;
    r = nr;
    nr = tmp;
  }
  if (t < 0) t += m;
  return (u64)t;
}

// w' = floor(w 2^64 / m) for Shoup multiplication.
u64 shoup_of(u64 w, u64 m) { return (u64)(((u128)w << 64) / m); }

ulonglong2 shoup_pair(u64 w, u64 m) {
  ulonglong2 r;
  r.x = w;
  r.y = shoup_of(w, m);
  return r;
}

bool miller_rabin(u64 n) {
  if (n < 2) return false;
  const u64 small[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 p : small)
    if (n % p == 0) return n == p;
  u64 d = n - 1;
  int s = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++s;
  }
  for (u64 a : small) {
    u64 x = powm(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int r = 1; r < s && witness; ++r) {
      x = mulm(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

// Primitive 2N-th root: smallest quadratic non-residue g >= 2, psi = g^((m-1)/2N).
u64 root_2n(u64 m, int logn) {
  u64 g = 2;
  while (powm(g, (m - 1) >> 1, m) != m - 1) ++g;
  return powm(g, (m - 1) >> (logn + 1), m);
}

unsigned brv(unsigned k, int bits) {
  unsigned r = 0;
  for (int i = 0; i < bits; ++i) {
    r = (r << 1) | (k & 1);
    k >>= 1;
  }
  return r;
}

// -m^-1 mod 2^64 by Newton iteration (m odd).
u64 neg_inv64(u64 m) {
  u64 x = m;  // correct to 3 bits
  for (int i = 0; i < 6; ++i) x *= 2 - m * x;
  return (u64)0 - x;
}

template <class F>
void par_for(int n, F f) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = std::max(1, std::min<int>(n, hw ? (int)hw : 4));
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (int i = t; i < n; i += nt) f(i);
    });
  for (auto &x : th) x.join();
}

}  // namespace

bool is_prime_u64(u64 n) { return miller_rabin(n); }

int build_tables(ks_context *c) {
  const int QP = c->qp, nq = c->nq, np = c->np, alpha = c->alpha, beta = c->beta;
  const int logn = c->logn, loga = c->loga, logb = c->logb, loggr = c->loggr;
  const size_t N = (size_t)1 << logn, N1 = (size_t)1 << loga, N2 = (size_t)1 << logb;
  const size_t GR = (size_t)1 << loggr;
  const size_t rowlen = (N2 - 1) * N1;
  const size_t twr_tile = (N2 - 1) * GR;  // entries per row tile

  std::vector<ModInfo> mod(QP);
  // (the inverse row pass reads the forward row table, mirrored: see ks_ntt.cuh)
  std::vector<ulonglong2> twc_f(QP * N1), twc_i(QP * N1), twr_f(QP * rowlen);
  std::vector<ulonglong2> iscale_q(nq), iscale_p(np), pinv(nq), pmod(nq);
  std::vector<u64> cup((size_t)beta * QP * alpha, 0), cdown((size_t)nq * alpha, 0);

  par_for(QP, [&](int t) {
    const u64 m = c->mods[t];
    ModInfo mi;
    mi.m = m;
    mi.minv = neg_inv64(m);
    mi.r1 = (u64)(((u128)1 << 64) % m);
    mi.r1s = shoup_of(mi.r1, m);
    mi.r2 = mulm(mi.r1, mi.r1, m);
    mi.mu = (u64)((((u128)1) << 64) / m);
    mod[t] = mi;
    const u64 psi = root_2n(m, logn);
    const u64 psi_inv = invm(psi, m);
    std::vector<u64> pw(N), pwi(N);
    pw[0] = pwi[0] = 1;
    for (size_t e = 1; e < N; ++e) {
      pw[e] = mulm(pw[e - 1], psi, m);
      pwi[e] = mulm(pwi[e - 1], psi_inv, m);
    }
    // Column table: entry k (1 <= k < N1) = psi^brv_logn(k).
    for (size_t k = 0; k < N1; ++k) {
      const unsigned e = brv((unsigned)k, logn);
      twc_f[t * N1 + k] = shoup_pair(k ? pw[e] : 1, m);
      twc_i[t * N1 + k] = shoup_pair(k ? pwi[e] : 1, m);
    }
    // Row table, by row tile b of GR rows (r = b*GR + g), stage-major inside a tile:
    // entry (b*(N2-1) + 2^ls - 1 + c)*GR + g = psi^brv_logn((N1 + r) 2^ls + c).
    for (size_t b = 0; b < N1 / GR; ++b)
      for (int ls = 0; ls < logb; ++ls)
        for (size_t cc = 0; cc < ((size_t)1 << ls); ++cc)
          for (size_t g = 0; g < GR; ++g) {
            const size_t r = b * GR + g;
            const size_t k = ((N1 + r) << ls) + cc;
            const unsigned e = brv((unsigned)k, logn);
            const size_t idx =
                t * rowlen + b * twr_tile + ((((size_t)1 << ls) - 1 + cc) << loggr) + g;
            twr_f[idx] = shoup_pair(pw[e], m);
          }
  });

  // iNTT scales: N^-1 * Qhat_{j,i}^-1 mod q_i for the digit j holding i.
  for (int i = 0; i < nq; ++i) {
    const u64 q = c->mods[i];
    const int j = i / alpha, lo = j * alpha, hi = std::min(nq, lo + alpha);
    u64 qhat = 1;
    for (int k = lo; k < hi; ++k)
      if (k != i) qhat = mulm(qhat, c->mods[k], q);
    const u64 s = mulm(invm(N % q, q), invm(qhat, q), q);
    iscale_q[i] = shoup_pair(s, q);
  }
  for (int k = 0; k < np; ++k) {
    const u64 p = c->mods[nq + k];
    u64 phat = 1;
    for (int kk = 0; kk < np; ++kk)
      if (kk != k) phat = mulm(phat, c->mods[nq + kk], p);
    iscale_p[k] = shoup_pair(mulm(invm(N % p, p), invm(phat, p), p), p);
  }
  // ModUp constants: (Qhat_{j,i} mod m_t) * 2^128 mod m_t (zero on the digit's own limbs).
  for (int j = 0; j < beta; ++j) {
    const int lo = j * alpha, hi = std::min(nq, lo + alpha);
    for (int t = 0; t < QP; ++t) {
      if (t >= lo && t < hi) continue;
      const u64 m = c->mods[t];
      for (int i = lo; i < hi; ++i) {
        u64 qhat = 1;
        for (int k = lo; k < hi; ++k)
          if (k != i) qhat = mulm(qhat, c->mods[k] % m, m);
        cup[((size_t)j * QP + t) * alpha + (i - lo)] = mulm(qhat, mod[t].r2, m);
      }
    }
  }
  // ModDown constants: (Phat_k mod q_i) * 2^64 mod q_i; P^-1 and P mod q_i.
  for (int i = 0; i < nq; ++i) {
    const u64 q = c->mods[i];
    u64 P = 1;
    for (int k = 0; k < np; ++k) {
      P = mulm(P, c->mods[nq + k] % q, q);
      u64 phat = 1;
      for (int kk = 0; kk < np; ++kk)
        if (kk != k) phat = mulm(phat, c->mods[nq + kk] % q, q);
      cdown[(size_t)i * alpha + k] = mulm(phat, mod[i].r1, q);
    }
    pinv[i] = shoup_pair(invm(P, q), q);
    pmod[i] = shoup_pair(P, q);
  }

  // Tensor-core basis conversion constants (ks_tc.cu): per (digit, target) / target, a
  // block [g < 2][k < ap][r < 8][a < 8] of bf16 values, the Toeplitz-shaped B operand:
  // entry (s = 8g + r, limb k, byte a) = byte s - a of the constant of source k (zero
  // outside bytes 0..7 and for missing sources), and in slot k = alpha the value 2^23
  // at a = 0 (it meets the 1.0 the A operand holds there, adding 2^23 to every sum).
  std::vector<u64> bup, bdown;
  if (c->tc_ap > 0) {
    const int ap = c->tc_ap;
    const size_t blk = 32 * (size_t)ap;  // words per block (256 ap bytes)
    auto bf16_byte = [](unsigned b) {
      const float f = (float)b;
      uint32_t bits;
      std::memcpy(&bits, &f, 4);
      return (uint16_t)(bits >> 16);
    };
    auto fill = [&](u64 *dst, const u64 *cst, int ns) {
      uint16_t *h = reinterpret_cast<uint16_t *>(dst);
      for (int g = 0; g < 2; ++g)
        for (int k = 0; k < ap; ++k)
          for (int r = 0; r < 8; ++r)
            for (int a = 0; a < 8; ++a) {
              const int sl = 8 * g + r, b = sl - a;
              uint16_t val = 0;
              if (k < ns && b >= 0 && b <= 7)
                val = bf16_byte((unsigned)(cst[k] >> (8 * b)) & 0xffu);
              else if (k == alpha && a == 0)
                val = 0x4B00;  // 2^23
              h[((g * ap + k) * 8 + r) * 8 + a] = val;
            }
    };
    bup.assign((size_t)beta * QP * blk, 0);
    bdown.assign((size_t)nq * blk, 0);
    for (int j = 0; j < beta; ++j) {
      const int lo = j * alpha, ns = std::min(nq, lo + alpha) - lo;
      for (int t = 0; t < QP; ++t)
        fill(&bup[((size_t)j * QP + t) * blk], &cup[((size_t)j * QP + t) * alpha], ns);
    }
    for (int i = 0; i < nq; ++i) fill(&bdown[(size_t)i * blk], &cdown[(size_t)i * alpha], np);
  }

  // One device allocation for everything (256-byte aligned pieces).
  struct Piece {
    const void *src;
    size_t bytes;
    void **dst;
  };
  Tables &T = c->tab;
  std::vector<Piece> pieces = {
      {mod.data(), mod.size() * sizeof(ModInfo), (void **)&T.mod},
      {twc_f.data(), twc_f.size() * 16, (void **)&T.twc_f},
      {twc_i.data(), twc_i.size() * 16, (void **)&T.twc_i},
      {twr_f.data(), twr_f.size() * 16, (void **)&T.twr_f},
      {iscale_q.data(), iscale_q.size() * 16, (void **)&T.iscale_q},
      {iscale_p.data(), iscale_p.size() * 16, (void **)&T.iscale_p},
      {cup.data(), cup.size() * 8, (void **)&T.cup},
      {cdown.data(), cdown.size() * 8, (void **)&T.cdown},
      {pinv.data(), pinv.size() * 16, (void **)&T.pinv},
      {pmod.data(), pmod.size() * 16, (void **)&T.pmod},
      {bup.data(), bup.size() * 8, (void **)&T.bup},
      {bdown.data(), bdown.size() * 8, (void **)&T.bdown},
      {nullptr, 256, (void **)&T.err},
  };
  size_t total = 0;
  for (auto &p : pieces) total += (p.bytes + 255) / 256 * 256;
  void *mem = nullptr;
  if (cudaMalloc(&mem, total) != cudaSuccess) {
    cudaGetLastError();
    return KS_ENOMEM;
  }
  std::vector<char> host(total, 0);
  size_t off = 0;
  for (auto &p : pieces) {
    if (p.src) std::memcpy(host.data() + off, p.src, p.bytes);
    *p.dst = (char *)mem + off;
    off += (p.bytes + 255) / 256 * 256;
  }
  if (cudaMemcpy(mem, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(mem);
    cudaGetLastError();
    return KS_ECUDA;
  }
  c->table_mem = mem;
  c->table_bytes = total;
  return KS_OK;
}

}  // namespace ks
