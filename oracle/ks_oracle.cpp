// Plain CPU oracle for the CKKS hybrid KeySwitch over RNS.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
// execute this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline / reference leg load it. It shares no code, header or table with
// the CUDA library.
//
// Everything here is schoolbook modular arithmetic: every reduction is an
// `unsigned __int128 %`, no Montgomery, Barrett or Shoup. The NTT is the
// recursive splitting of x^M - zeta into x^{M/2} -+ sqrt(zeta) (written from
// the definition of the negacyclic transform, not from any GPU dataflow).
//
// Paper: "Dataflow-Oriented Classification and Performance Analysis of
// GPU-Accelerated Homomorphic Encryption", Sec. II-A (CKKS and KeySwitch),
// Fig. 1 (KeySwitch: iNTT -> BConv -> NTT, key multiply, iNTT -> BConv -> NTT).
// Readings where the paper is silent (ring x^N+1, L+1 primes, ceil alpha,
// bit-reversed NTT order, uncorrected BConv, floor ModDown) are listed in the
// design notes and restated at each function below.
//
// Parity status: every function below is pinned by tests/test_oracle_*.py
// (direct evaluation, schoolbook convolution, big-integer CRT, special cases,
// noise bound). No function is "parity unpinned".

#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <algorithm>

typedef unsigned __int128 u128;
typedef uint64_t u64;

namespace {

u64 mmul(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
u64 madd(u64 a, u64 b, u64 m) { return (u64)(((u128)a + b) % m); }
u64 msub(u64 a, u64 b, u64 m) { return (u64)(((u128)a + m - (b % m)) % m); }

u64 mpow(u64 b, u64 e, u64 m) {
  u64 r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = mmul(r, b, m);
    b = mmul(b, b, m);
    e >>= 1;
  }
  return r;
}

// Inverse modulo a prime by Fermat's little theorem.
u64 minv(u64 a, u64 p) { return mpow(a, p - 2, p); }

// Deterministic Miller-Rabin for 64-bit inputs with the first 12 prime bases.
bool is_prime(u64 n) {
  if (n < 2) return false;
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 b : bases) {
    if (n == b) return true;
    if (n % b == 0) return false;
  }
  u64 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (u64 a : bases) {
    u64 x = mpow(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = mmul(x, x, n);
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

// Primitive 2N-th root of unity: psi = g^((q-1)/2N) with g the smallest
// integer >= 2 that is a quadratic non-residue (g^((q-1)/2) = -1).
u64 find_psi(u64 q, int logn) {
  u64 g = 2;
  while (mpow(g, (q - 1) / 2, q) != q - 1) ++g;
  return mpow(g, (q - 1) >> (logn + 1), q);
}

// Run f(i) for i in [0, n) on up to nthreads threads.
template <class F>
void parallel_for(int n, int nthreads, F f) {
  if (nthreads <= 1 || n <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  int nt = std::min(nthreads, n);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (int i = t; i < n; i += nt) f(i);
    });
  for (auto &x : th) x.join();
}

// Powers psi^e for e in [0, 2N).
std::vector<u64> psi_powers(u64 q, int logn) {
  u64 n2 = (u64)2 << logn;
  u64 psi = find_psi(q, logn);
  std::vector<u64> pw(n2);
  pw[0] = 1;
  for (u64 e = 1; e < n2; ++e) pw[e] = mmul(pw[e - 1], psi, q);
  return pw;
}

// Negacyclic NTT, by definition: a(x) mod (x^M - psi^e) splits into
// a mod (x^{M/2} - psi^{e/2}) (first half of the output) and
// a mod (x^{M/2} + psi^{e/2}) = a mod (x^{M/2} - psi^{e/2 + N}) (second half).
// At M = 1 the remainder is the evaluation a(psi^e). Started with
// x^N + 1 = x^N - psi^N, this yields the evaluations at the odd powers of psi
// in bit-reversed order: slot k holds a(psi^(2*brv(k)+1)).
void ntt_rec(u64 *a, u64 M, u64 e, u64 N, u64 q, const std::vector<u64> &pw) {
  if (M == 1) return;
  u64 h = M / 2;
  u64 z = pw[(e / 2) % (2 * N)];
  for (u64 j = 0; j < h; ++j) {
    u64 t = mmul(z, a[j + h], q);
    u64 lo = madd(a[j], t, q);
    u64 hi = msub(a[j], t, q);
    a[j] = lo;
    a[j + h] = hi;
  }
  ntt_rec(a, h, e / 2, N, q, pw);
  ntt_rec(a + h, h, (e / 2 + N) % (2 * N), N, q, pw);
}

// Exact inverse of ntt_rec: undo the two halves, then rebuild
// a_lo = (lo + hi)/2 and a_hi = (lo - hi)/(2z).
void intt_rec(u64 *a, u64 M, u64 e, u64 N, u64 q, const std::vector<u64> &pw,
              u64 inv2) {
  if (M == 1) return;
  u64 h = M / 2;
  intt_rec(a, h, e / 2, N, q, pw, inv2);
  intt_rec(a + h, h, (e / 2 + N) % (2 * N), N, q, pw, inv2);
  u64 zinv = pw[(2 * N - (e / 2) % (2 * N)) % (2 * N)];
  u64 c = mmul(inv2, zinv, q);
  for (u64 j = 0; j < h; ++j) {
    u64 lo = a[j], hi = a[j + h];
    a[j] = mmul(madd(lo, hi, q), inv2, q);
    a[j + h] = mmul(msub(lo, hi, q), c, q);
  }
}

void ntt_fwd(u64 *a, int logn, u64 q, const std::vector<u64> &pw) {
  u64 N = (u64)1 << logn;
  for (u64 i = 0; i < N; ++i) a[i] %= q;
  ntt_rec(a, N, N, N, q, pw);
}

void ntt_inv(u64 *a, int logn, u64 q, const std::vector<u64> &pw) {
  u64 N = (u64)1 << logn;
  for (u64 i = 0; i < N; ++i) a[i] %= q;
  intt_rec(a, N, N, N, q, pw, (q + 1) / 2);
}

// Fast (uncorrected) basis conversion, Sec. II-A ("BConv converts a
// polynomial into an approximately equivalent polynomial with a different set
// of moduli"). For sources {s_i} with S = prod s_i and S_i = S / s_i:
//   y_t[n] = sum_i [x_i[n] * S_i^{-1}]_{s_i} * (S_i mod m_t)   (mod m_t)
// which is X mod m_t for the integer X = x + u*S, 0 <= u < #sources.
void bconv(const u64 *const *x, const u64 *src, int ns, const u64 *dst, int nd,
           u64 *const *y, u64 N, int nthreads) {
  std::vector<u64> sinv(ns);
  for (int i = 0; i < ns; ++i) {
    u64 shat = 1;
    for (int k = 0; k < ns; ++k)
      if (k != i) shat = mmul(shat, src[k], src[i]);
    sinv[i] = minv(shat, src[i]);
  }
  parallel_for(nd, nthreads, [&](int t) {
    u64 m = dst[t];
    std::vector<u64> shat_t(ns);
    for (int i = 0; i < ns; ++i) {
      u64 s = 1;
      for (int k = 0; k < ns; ++k)
        if (k != i) s = mmul(s, src[k], m);
      shat_t[i] = s;
    }
    for (u64 n = 0; n < N; ++n) {
      u64 acc = 0;
      for (int i = 0; i < ns; ++i) {
        u64 v = mmul(x[i][n], sinv[i], src[i]);
        acc = madd(acc, mmul(v, shat_t[i], m), m);
      }
      y[t][n] = acc;
    }
  });
}

struct Basis {
  int logn, L, dnum, alpha, beta, nq, np, qp;
  u64 N;
  std::vector<u64> mod;                 // QP moduli: q_0..q_L, p_0..p_{alpha-1}
  std::vector<std::vector<u64>> pw;     // psi powers per modulus
};

int make_basis(Basis &B, int dnum, int logn, int L, const u64 *q, int nq,
               const u64 *p, int np, int nthreads) {
  if (dnum < 1 || logn < 1 || logn > 17 || L < 0 || nq != L + 1) return -1;
  B.dnum = dnum; B.logn = logn; B.L = L;
  B.N = (u64)1 << logn;
  B.nq = nq;
  // alpha = ceil((L+1)/dnum), Table I; digits beta = ceil((L+1)/alpha).
  B.alpha = (L + 1 + dnum - 1) / dnum;
  B.beta = (L + 1 + B.alpha - 1) / B.alpha;
  if (np != B.alpha) return -1;
  B.np = np;
  B.qp = nq + np;
  B.mod.assign(q, q + nq);
  B.mod.insert(B.mod.end(), p, p + np);
  B.pw.resize(B.qp);
  parallel_for(B.qp, nthreads, [&](int t) { B.pw[t] = psi_powers(B.mod[t], logn); });
  return 0;
}

// Digit j covers Q-limbs [j*alpha, min((j+1)*alpha, L+1)).
int digit_lo(const Basis &B, int j) { return j * B.alpha; }
int digit_hi(const Basis &B, int j) { return std::min((j + 1) * B.alpha, B.nq); }

}  // namespace

extern "C" {

int orc_is_prime(u64 n) { return is_prime(n) ? 1 : 0; }

u64 orc_find_psi(u64 q, int logn) { return find_psi(q, logn); }

// In-place forward / inverse negacyclic NTT of `count` limbs a[count][N],
// limb c modulo mods[c].
void orc_ntt_fwd(u64 *a, const u64 *mods, int count, int logn, int nthreads) {
  u64 N = (u64)1 << logn;
  parallel_for(count, nthreads, [&](int c) {
    auto pw = psi_powers(mods[c], logn);
    ntt_fwd(a + (size_t)c * N, logn, mods[c], pw);
  });
}

void orc_ntt_inv(u64 *a, const u64 *mods, int count, int logn, int nthreads) {
  u64 N = (u64)1 << logn;
  parallel_for(count, nthreads, [&](int c) {
    auto pw = psi_powers(mods[c], logn);
    ntt_inv(a + (size_t)c * N, logn, mods[c], pw);
  });
}

// Fast basis conversion of coefficient-form limbs x[ns][N] (mod src) onto
// dst: y[nd][N].
void orc_bconv(const u64 *x, const u64 *src, int ns, const u64 *dst, int nd,
               u64 *y, int logn, int nthreads) {
  u64 N = (u64)1 << logn;
  std::vector<const u64 *> xp(ns);
  std::vector<u64 *> yp(nd);
  for (int i = 0; i < ns; ++i) xp[i] = x + (size_t)i * N;
  for (int t = 0; t < nd; ++t) yp[t] = y + (size_t)t * N;
  bconv(xp.data(), src, ns, dst, nd, yp.data(), N, nthreads);
}

}  // extern "C"

namespace {

// ModDown (second phase of Fig. 1) at level l of basis B: acc[l+1+alpha][N] in NTT
// form over q_0..q_l, p_0..p_{alpha-1} -> out[l+1][N] in NTT form over q_0..q_l:
//   out = (acc - NTT(BConv_{P->Q_l}(iNTT(acc_P)))) * P^{-1}.
// Floor variant (no +P/2 rounding).
void moddown_at(const Basis &B, int level, const u64 *acc, u64 *out, int nthreads) {
  const u64 N = B.N;
  const int nq = level + 1, np = B.np, logn = B.logn;
  const u64 *q = B.mod.data(), *p = B.mod.data() + B.nq;
  std::vector<u64> cp((size_t)np * N);
  std::memcpy(cp.data(), acc + (size_t)nq * N, cp.size() * 8);
  parallel_for(np, nthreads, [&](int k) {
    ntt_inv(cp.data() + (size_t)k * N, logn, p[k], B.pw[B.nq + k]);
  });
  std::vector<u64> z((size_t)nq * N);
  std::vector<const u64 *> xp(np);
  std::vector<u64 *> yp(nq);
  for (int k = 0; k < np; ++k) xp[k] = cp.data() + (size_t)k * N;
  for (int i = 0; i < nq; ++i) yp[i] = z.data() + (size_t)i * N;
  bconv(xp.data(), p, np, q, nq, yp.data(), N, nthreads);
  parallel_for(nq, nthreads, [&](int i) {
    u64 *zi = z.data() + (size_t)i * N;
    ntt_fwd(zi, logn, q[i], B.pw[i]);
    u64 P = 1;
    for (int k = 0; k < np; ++k) P = mmul(P, p[k], q[i]);
    u64 Pinv = minv(P, q[i]);
    const u64 *ai = acc + (size_t)i * N;
    u64 *oi = out + (size_t)i * N;
    for (u64 n = 0; n < N; ++n) oi[n] = mmul(msub(ai[n], zi[n], q[i]), Pinv, q[i]);
  });
}

// Hybrid KeySwitch (Sec. II-A, Fig. 1) at level l <= L of basis B (built for level L).
// At level l the input has l+1 limbs, the digits are D_j = [j alpha, min((j+1) alpha,
// l+1)) with the top level's alpha, beta_l = ceil((l+1)/alpha), and the key is the
// top level's: evk[beta][2][QP][N] whose limb t of Q_l is row t and whose P-limb k
// is row L+1+k (its other rows belong to the dropped primes and are not read).
//   d [l+1][N], out [2][l+1][N]; traces ext [beta_l][l+1+alpha][N], acc [2][l+1+alpha][N].
void keyswitch_at(const Basis &B, int level, const u64 *d, const u64 *evk, u64 *out,
                  u64 *ext_trace, u64 *acc_trace, int nthreads) {
  const u64 N = B.N;
  const int logn = B.logn, nq = level + 1, alpha = B.alpha;
  const int QP = nq + alpha, beta = (nq + alpha - 1) / alpha;
  // moduli of level l: q_0..q_l then p_0..p_{alpha-1}; their rows in B and in evk
  std::vector<int> row(QP);
  for (int t = 0; t < QP; ++t) row[t] = t < nq ? t : B.nq + (t - nq);
  std::vector<u64> mod(QP);
  for (int t = 0; t < QP; ++t) mod[t] = B.mod[row[t]];
  // Step 1: iNTT of the l+1 input limbs.
  std::vector<u64> x((size_t)nq * N);
  std::memcpy(x.data(), d, x.size() * 8);
  parallel_for(nq, nthreads, [&](int i) {
    ntt_inv(x.data() + (size_t)i * N, logn, mod[i], B.pw[i]);
  });
  // Steps 2-4: per digit, ModUp = BConv onto (Q_l u P) \ D_j then NTT; the
  // digit's own limbs are the input limbs themselves.
  std::vector<u64> ext((size_t)beta * QP * N);
  for (int j = 0; j < beta; ++j) {
    const int lo = j * alpha, hi = std::min((j + 1) * alpha, nq);
    std::vector<u64> src(mod.begin() + lo, mod.begin() + hi);
    std::vector<int> tgt;
    for (int t = 0; t < QP; ++t)
      if (t < lo || t >= hi) tgt.push_back(t);
    std::vector<u64> dst;
    for (int t : tgt) dst.push_back(mod[t]);
    u64 *ej = ext.data() + (size_t)j * QP * N;
    std::vector<const u64 *> xp;
    for (int i = lo; i < hi; ++i) xp.push_back(x.data() + (size_t)i * N);
    std::vector<u64 *> yp;
    for (int t : tgt) yp.push_back(ej + (size_t)t * N);
    bconv(xp.data(), src.data(), (int)src.size(), dst.data(), (int)dst.size(),
          yp.data(), N, nthreads);
    parallel_for((int)tgt.size(), nthreads, [&](int k) {
      int t = tgt[k];
      ntt_fwd(ej + (size_t)t * N, logn, mod[t], B.pw[row[t]]);
    });
    for (int i = lo; i < hi; ++i)
      std::memcpy(ej + (size_t)i * N, d + (size_t)i * N, N * 8);
  }
  // Step 5: key multiply, accumulated over the digits.
  std::vector<u64> acc((size_t)2 * QP * N);
  parallel_for(2 * QP, nthreads, [&](int ct) {
    int c = ct / QP, t = ct % QP;
    u64 m = mod[t];
    u64 *a = acc.data() + ((size_t)c * QP + t) * N;
    for (u64 n = 0; n < N; ++n) {
      u64 s = 0;
      for (int j = 0; j < beta; ++j) {
        u64 e = ext[((size_t)j * QP + t) * N + n];
        u64 k = evk[(((size_t)j * 2 + c) * B.qp + row[t]) * N + n];
        s = madd(s, mmul(e, k, m), m);
      }
      a[n] = s;
    }
  });
  // Steps 6-8: ModDown of both polynomials.
  for (int c = 0; c < 2; ++c)
    moddown_at(B, level, acc.data() + (size_t)c * QP * N, out + (size_t)c * nq * N, nthreads);
  if (ext_trace) std::memcpy(ext_trace, ext.data(), ext.size() * 8);
  if (acc_trace) std::memcpy(acc_trace, acc.data(), acc.size() * 8);
}

// The automorphism sigma_k(a)(x) = a(x^k) of one coefficient-form limb mod m:
// x^n goes to x^(nk mod 2N), and x^e = -x^(e-N) for e >= N (x^N = -1).
void automorphism(const u64 *a, u64 *out, u64 N, u64 k, u64 m) {
  for (u64 n = 0; n < N; ++n) {
    u64 e = (n * k) % (2 * N);
    if (e < N) out[e] = a[n];
    else out[e - N] = a[n] ? m - a[n] : 0;
  }
}

}  // namespace

extern "C" {

// ModDown of acc[QP][N] at the top level L (see moddown_at).
int orc_moddown(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p,
                int np, const u64 *acc, u64 *out, int nthreads) {
  Basis B;
  if (make_basis(B, dnum, logn, L, q, nq, p, np, nthreads)) return -1;
  moddown_at(B, L, acc, out, nthreads);
  return 0;
}

// Hybrid KeySwitch (Sec. II-A, Fig. 1) at level L.
//   d   [L+1][N]           input polynomial, NTT form, limb i mod q_i
//   evk [beta][2][QP][N]   key pairs (b_j, a_j), NTT form over Q u P
//   out [2][L+1][N]        switched pair, NTT form over Q
// Optional traces (may be null): ext [beta][QP][N] (ModUp output, NTT form),
// acc [2][QP][N] (key-multiply output, NTT form).
int orc_keyswitch(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p,
                  int np, const u64 *d, const u64 *evk, u64 *out, u64 *ext_trace,
                  u64 *acc_trace, int nthreads) {
  Basis B;
  if (make_basis(B, dnum, logn, L, q, nq, p, np, nthreads)) return -1;
  keyswitch_at(B, L, d, evk, out, ext_trace, acc_trace, nthreads);
  return 0;
}

// KeySwitch at level `level` (0..L) with the key of the level-L basis (see
// keyswitch_at): d [level+1][N], out [2][level+1][N].
int orc_keyswitch_level(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p,
                        int np, int level, const u64 *d, const u64 *evk, u64 *out,
                        int nthreads) {
  Basis B;
  if (make_basis(B, dnum, logn, L, q, nq, p, np, nthreads)) return -1;
  if (level < 0 || level > L) return -1;
  keyswitch_at(B, level, d, evk, out, nullptr, nullptr, nthreads);
  return 0;
}

// HMUL (Sec. II-A) at level `level`: ct1 = (x0, x1), ct2 = (y0, y1), each
// [2][level+1][N] in NTT form over Q_level:
//   out = (x0 y0, x0 y1 + x1 y0) + KS(x1 y1)   (no rescaling)
// with KS under the relinearisation key rlk (s_from = s^2, s_to = s) of the level-L basis.
int orc_hmul(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p, int np,
             int level, const u64 *ct1, const u64 *ct2, const u64 *rlk, u64 *out,
             int nthreads) {
  Basis B;
  if (make_basis(B, dnum, logn, L, q, nq, p, np, nthreads)) return -1;
  if (level < 0 || level > L) return -1;
  const u64 N = B.N;
  const size_t P = (size_t)(level + 1) * N;
  std::vector<u64> d2(P), ks(2 * P);
  std::vector<u64> t0(P), t1(P);
  for (int i = 0; i <= level; ++i) {
    const u64 m = q[i];
    for (u64 n = 0; n < N; ++n) {
      const size_t k = (size_t)i * N + n;
      const u64 x0 = ct1[k], x1 = ct1[P + k], y0 = ct2[k], y1 = ct2[P + k];
      t0[k] = mmul(x0, y0, m);
      t1[k] = madd(mmul(x0, y1, m), mmul(x1, y0, m), m);
      d2[k] = mmul(x1, y1, m);
    }
  }
  keyswitch_at(B, level, d2.data(), rlk, ks.data(), nullptr, nullptr, nthreads);
  for (int i = 0; i <= level; ++i)
    for (u64 n = 0; n < N; ++n) {
      const size_t k = (size_t)i * N + n;
      out[k] = madd(t0[k], ks[k], q[i]);
      out[P + k] = madd(t1[k], ks[P + k], q[i]);
    }
  return 0;
}

// Galois automorphism x -> x^k (k odd) of limbs a[count][N] in NTT form mod mods[c]:
// inverse NTT, the coefficient map of `automorphism`, forward NTT.
void orc_automorph_ntt(const u64 *a, u64 *out, const u64 *mods, int count, int logn, u64 k,
                       int nthreads) {
  const u64 N = (u64)1 << logn;
  parallel_for(count, nthreads, [&](int c) {
    auto pw = psi_powers(mods[c], logn);
    std::vector<u64> x(a + (size_t)c * N, a + (size_t)(c + 1) * N);
    ntt_inv(x.data(), logn, mods[c], pw);
    automorphism(x.data(), out + (size_t)c * N, N, k, mods[c]);
    ntt_fwd(out + (size_t)c * N, logn, mods[c], pw);
  });
}

// HROT (Sec. II-A) at level `level`: ct = (c0, c1) [2][level+1][N] NTT form,
//   out = (sigma_k(c0), 0) + KS(sigma_k(c1))
// with KS under the rotation key rtk (s_from = sigma_k(s), s_to = s).
int orc_hrot(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p, int np,
             int level, const u64 *ct, u64 k, const u64 *rtk, u64 *out, int nthreads) {
  Basis B;
  if (make_basis(B, dnum, logn, L, q, nq, p, np, nthreads)) return -1;
  if (level < 0 || level > L || (k & 1) == 0 || k >= 2 * B.N) return -1;
  const u64 N = B.N;
  const size_t P = (size_t)(level + 1) * N;
  std::vector<u64> r(2 * P), ks(2 * P);
  orc_automorph_ntt(ct, r.data(), q, level + 1, logn, k, nthreads);
  orc_automorph_ntt(ct + P, r.data() + P, q, level + 1, logn, k, nthreads);
  keyswitch_at(B, level, r.data() + P, rtk, ks.data(), nullptr, nullptr, nthreads);
  for (int i = 0; i <= level; ++i)
    for (u64 n = 0; n < N; ++n) {
      const size_t kk = (size_t)i * N + n;
      out[kk] = madd(r[kk], ks[kk], q[i]);
      out[P + kk] = ks[P + kk];
    }
  return 0;
}

// Product of two integer polynomials mod x^N + 1 (schoolbook, negacyclic wrap);
// used for s^2 of a small key. |coefficients| stay far below 2^63 for keys.
void orc_negacyclic_mul_i64(const int64_t *a, const int64_t *b, int64_t *out, int logn) {
  const int64_t N = (int64_t)1 << logn;
  for (int64_t n = 0; n < N; ++n) out[n] = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (a[i] == 0) continue;
    for (int64_t j = 0; j < N; ++j) {
      const int64_t v = a[i] * b[j];
      if (i + j < N) out[i + j] += v;
      else out[i + j - N] -= v;
    }
  }
}

// sigma_k of an integer polynomial (coefficient form).
void orc_automorphism_i64(const int64_t *a, int64_t *out, int logn, u64 k) {
  const u64 N = (u64)1 << logn;
  for (u64 n = 0; n < N; ++n) {
    u64 e = (n * k) % (2 * N);
    if (e < N) out[e] = a[n];
    else out[e - N] = -a[n];
  }
}

// Evaluation-key generation from given randomness (the method's random draws
// are inputs): for each digit j,
//   evk_j = (b_j, a_j),  b_j = -a_j*s_to + e_j + [P*g_j]*s_from   over Q u P,
// where g_j = 1 mod the primes of D_j and 0 mod every other prime, so
// [P*g_j]_{q_i} = P mod q_i for i in D_j, else 0; and [P*g_j]_{p_k} = 0.
//   s_from, s_to [N] ternary, a [beta][QP][N] NTT form, e [beta][N] small ints.
int orc_keygen_poly(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p,
                    int np, const int64_t *s_from, const int8_t *s_to, const u64 *a,
                    const int32_t *e, u64 *evk, int nthreads);

int orc_keygen(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p,
               int np, const int8_t *s_from, const int8_t *s_to, const u64 *a,
               const int32_t *e, u64 *evk, int nthreads) {
  if (logn < 1 || logn > 17) return -1;
  std::vector<int64_t> sf(s_from, s_from + ((size_t)1 << logn));
  return orc_keygen_poly(dnum, logn, L, q, nq, p, np, sf.data(), s_to, a, e, evk, nthreads);
}

// As orc_keygen with s_from any integer polynomial (|s_from[n]| < 2^62): the
// relinearisation key takes s_from = s^2, a rotation key s_from = sigma_k(s).
int orc_keygen_poly(int dnum, int logn, int L, const u64 *q, int nq, const u64 *p,
                    int np, const int64_t *s_from, const int8_t *s_to, const u64 *a,
                    const int32_t *e, u64 *evk, int nthreads) {
  Basis B;
  if (make_basis(B, dnum, logn, L, q, nq, p, np, nthreads)) return -1;
  const u64 N = B.N;
  const int QP = B.qp;
  parallel_for(QP, nthreads, [&](int t) {
    u64 m = B.mod[t];
    std::vector<u64> sf(N), st(N), ej(N);
    for (u64 n = 0; n < N; ++n) {
      sf[n] = s_from[n] >= 0 ? (u64)s_from[n] % m : msub(0, (u64)(-s_from[n]) % m, m);
      st[n] = s_to[n] >= 0 ? (u64)s_to[n] : m - (u64)(-s_to[n]);
    }
    ntt_fwd(sf.data(), logn, m, B.pw[t]);
    ntt_fwd(st.data(), logn, m, B.pw[t]);
    u64 P = 1;
    for (int k = 0; k < np; ++k) P = mmul(P, p[k], m);
    for (int j = 0; j < B.beta; ++j) {
      const int32_t *ev = e + (size_t)j * N;
      for (u64 n = 0; n < N; ++n)
        ej[n] = ev[n] >= 0 ? (u64)ev[n] % m : msub(0, (u64)(-(int64_t)ev[n]) % m, m);
      ntt_fwd(ej.data(), logn, m, B.pw[t]);
      bool in_digit = t < nq && t >= digit_lo(B, j) && t < digit_hi(B, j);
      u64 g = in_digit ? P : 0;
      const u64 *aj = a + ((size_t)j * QP + t) * N;
      u64 *bj = evk + (((size_t)j * 2 + 0) * QP + t) * N;
      u64 *a_out = evk + (((size_t)j * 2 + 1) * QP + t) * N;
      for (u64 n = 0; n < N; ++n) {
        u64 v = msub(ej[n], mmul(aj[n], st[n], m), m);
        v = madd(v, mmul(g, sf[n], m), m);
        bj[n] = v;
        a_out[n] = aj[n] % m;
      }
    }
  });
  return 0;
}

}  // extern "C"
