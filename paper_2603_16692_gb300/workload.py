"""Seeded synthetic workloads for the KeySwitch: parameters, primes, inputs, key material.

This module only draws numbers. It holds none of the KeySwitch arithmetic, and it
serves both the CUDA path and the CPU oracle with the same inputs.

Recipe (the paper uses no dataset; its workload is synthetic HMUL timing over a
(dnum, N, L) grid, Sec. IV-A):

* primes: q_0..q_L are the L+1 largest primes below 2^50 with q = 1 mod 2N, in
  descending order; p_0..p_{alpha-1} are the alpha largest primes below 2^60 with
  p = 1 mod 2N. alpha = ceil((L+1)/dnum) (Table I), beta = ceil((L+1)/alpha).
* d: uniform residues mod each q_i, taken as the NTT-form input polynomial.
* keys: s_from, s_to ternary, each coefficient uniform in {-1, 0, 1}.
* a: uniform residues mod each of the QP primes (NTT form).
* e: rounded Gaussian with sigma = 3.2, cut at |e| <= 19.
All draws use numpy's PCG64 keyed by the seed.
"""
from __future__ import annotations

import dataclasses
import functools

import numpy as np

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def _probable_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 2^64 (first 12 prime bases)."""
    if n < 2:
        return False
    for b in _MR_BASES:
        if n % b == 0:
            return n == b
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


@functools.lru_cache(maxsize=None)
def primes_below(bits: int, logn: int, count: int) -> tuple:
    """The `count` largest primes p < 2^bits with p = 1 mod 2^(logn+1), descending."""
    step = 1 << (logn + 1)
    c = ((1 << bits) - 1) // step * step + 1
    if c >= (1 << bits):
        c -= step
    out = []
    while len(out) < count:
        if c < step:
            raise ValueError("not enough primes")
        if _probable_prime(c):
            out.append(c)
        c -= step
    return tuple(out)


@dataclasses.dataclass(frozen=True)
class Params:
    dnum: int
    logn: int
    L: int
    q: tuple
    p: tuple

    @property
    def N(self) -> int:
        return 1 << self.logn

    @property
    def alpha(self) -> int:
        return -(-(self.L + 1) // self.dnum)

    @property
    def beta(self) -> int:
        return -(-(self.L + 1) // self.alpha)

    @property
    def QP(self) -> int:
        return self.L + 1 + self.alpha

    @property
    def mods(self) -> tuple:
        return tuple(self.q) + tuple(self.p)

    def digit(self, j: int) -> range:
        return range(j * self.alpha, min((j + 1) * self.alpha, self.L + 1))

    def name(self) -> str:
        return f"({self.dnum},2^{self.logn},{self.L})"

    # algorithmic HBM bytes of one KeySwitch: read d, read evk, write out
    def algo_bytes(self) -> int:
        n = self.N * 8
        return (self.L + 1) * n + 2 * self.beta * self.QP * n + 2 * (self.L + 1) * n


def make_params(dnum: int, logn: int, L: int, qbits: int = 50, pbits: int = 60) -> Params:
    alpha = -(-(L + 1) // dnum)
    q = primes_below(qbits, logn, L + 1)
    p = primes_below(pbits, logn, alpha)
    return Params(dnum, logn, L, q, p)


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, stream]))


def uniform_limbs(g: np.random.Generator, mods, n: int) -> np.ndarray:
    out = np.empty((len(mods), n), dtype=np.uint64)
    for i, m in enumerate(mods):
        out[i] = g.integers(0, m, size=n, dtype=np.uint64)
    return out


def gen_input(prm: Params, seed: int) -> np.ndarray:
    """d[L+1][N]: uniform mod each q_i (NTT form)."""
    return uniform_limbs(rng(seed, 1), prm.q, prm.N)


def gen_keys(prm: Params, seed: int):
    """(s_from, s_to, a, e): ternary keys [N] int8, a[beta][QP][N] uint64, e[beta][N] int32."""
    g = rng(seed, 2)
    s_from = g.integers(-1, 2, size=prm.N, dtype=np.int8)
    s_to = g.integers(-1, 2, size=prm.N, dtype=np.int8)
    a = np.stack([uniform_limbs(g, prm.mods, prm.N) for _ in range(prm.beta)])
    e = np.empty((prm.beta, prm.N), dtype=np.int32)
    for j in range(prm.beta):
        while True:
            v = np.rint(g.normal(0.0, 3.2, size=prm.N))
            if np.all(np.abs(v) <= 19):
                break
        e[j] = v.astype(np.int32)
    return s_from, s_to, a, e


# The workloads the benchmark and the parity tests use.
C1 = (2, 13, 7)      # (dnum, log2 N, L)
C2 = (2, 15, 10)
C3 = (4, 16, 35)


def batch_jobs(seed: int, count: int = 64):
    """Uneven (dnum, log2N, L) jobs: N in 2^13..2^17, L in [4, 60], dnum in [2, 10]."""
    g = rng(seed, 3)
    jobs = []
    for _ in range(count):
        logn = int(g.integers(13, 18))
        L = int(g.integers(4, 61))
        dnum = int(g.integers(2, 11))
        jobs.append((dnum, logn, L))
    return jobs


def selector_points(seed: int = 0, count: int = 200):
    """Seeded (dnum, log2N, L) points for the selector sweep, over the batch ranges;
    the largest workload (10, 2^17, 60) is always included."""
    g = rng(seed, 4)
    pts = [(10, 17, 60)]
    while len(pts) < count:
        p = (int(g.integers(2, 11)), int(g.integers(13, 18)), int(g.integers(4, 61)))
        if p not in pts:
            pts.append(p)
    return pts
