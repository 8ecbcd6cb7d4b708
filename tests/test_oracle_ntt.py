"""Pins of the oracle's primes, roots and negacyclic NTT (CPU only).

The NTT convention (ring x^N + 1, slot k = a(psi^(2 brv(k) + 1))) is the
reading taken for the transform that Sec. II-A names but does not define.
"""
import numpy as np
import pytest
import sympy

from oracle import oracle as O
from paper_2603_16692_gb300 import workload as W
from tests import pins


@pytest.mark.parametrize("logn", [1, 4, 6, 13, 17])
def test_generated_primes_are_ntt_friendly(logn):
    for bits in (50, 60):
        ps = W.primes_below(bits, logn, 6)
        assert len(set(ps)) == 6 and list(ps) == sorted(ps, reverse=True)
        for p in ps:
            assert p < (1 << bits) and p % (1 << (logn + 1)) == 1
            assert sympy.isprime(p) and O.is_prime(p)
        # no prime of the form was skipped between consecutive picks
        step = 1 << (logn + 1)
        for a, b in zip(ps, ps[1:]):
            for c in range(b + step, a, step):
                assert not sympy.isprime(c)


def test_oracle_primality_matches_sympy():
    g = np.random.default_rng(7)
    cases = [0, 1, 2, 3, 4, 561, 1105, 3215031751, 2152302898747, 3474749660383,
             341550071728321, 3825123056546413051, 318665857834031151167461 % (1 << 64),
             (1 << 61) - 1, (1 << 64) - 59, (1 << 64) - 1]
    cases += [int(x) for x in g.integers(0, 1 << 62, size=300, dtype=np.uint64)]
    cases += [int(x) | 1 for x in g.integers(1 << 40, 1 << 50, size=300, dtype=np.uint64)]
    for n in cases:
        assert O.is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("logn", [1, 3, 8, 13, 16, 17])
def test_psi_is_primitive_2n_root(logn):
    for q in W.primes_below(50, logn, 2) + W.primes_below(60, logn, 2):
        psi = O.find_psi(q, logn)
        n = 1 << logn
        assert pow(psi, n, q) == q - 1          # psi^N = -1  => order exactly 2N
        assert pow(psi, 2 * n, q) == 1
        # smallest non-residue rule: every g in [2, g0) is a residue
        g0 = 2
        while pow(g0, (q - 1) // 2, q) != q - 1:
            g0 += 1
        assert psi == pow(g0, (q - 1) // (2 * n), q)


@pytest.mark.parametrize("logn", [1, 2, 3, 4, 5, 6])
def test_ntt_equals_direct_evaluation(logn):
    g = np.random.default_rng(logn)
    for q in (W.primes_below(50, logn, 1)[0], W.primes_below(60, logn, 1)[0]):
        a = g.integers(0, q, size=(1, 1 << logn), dtype=np.uint64)
        got = O.ntt_fwd(a, [q], logn)[0]
        want = pins.ntt_direct(a[0], q, O.find_psi(q, logn), logn)
        assert [int(x) for x in got] == want


@pytest.mark.parametrize("logn", [1, 3, 5, 6])
def test_ntt_product_is_negacyclic_convolution(logn):
    g = np.random.default_rng(100 + logn)
    q = W.primes_below(50, logn, 1)[0]
    a = g.integers(0, q, size=(1, 1 << logn), dtype=np.uint64)
    b = g.integers(0, q, size=(1, 1 << logn), dtype=np.uint64)
    ah, bh = O.ntt_fwd(a, [q], logn), O.ntt_fwd(b, [q], logn)
    prod = np.array([[int(x) * int(y) % q for x, y in zip(ah[0], bh[0])]], dtype=np.uint64)
    c = O.ntt_inv(prod, [q], logn)[0]
    assert [int(x) for x in c] == pins.negacyclic_mul(a[0], b[0], q)


@pytest.mark.parametrize("logn", list(range(1, 18)))
def test_ntt_roundtrip(logn):
    g = np.random.default_rng(200 + logn)
    mods = list(W.primes_below(50, logn, 2)) + list(W.primes_below(60, logn, 1))
    a = np.stack([g.integers(0, m, size=1 << logn, dtype=np.uint64) for m in mods])
    f = O.ntt_fwd(a, mods, logn)
    assert np.array_equal(O.ntt_inv(f, mods, logn), a)
    assert np.array_equal(O.ntt_fwd(O.ntt_inv(a, mods, logn), mods, logn), a)
    assert all(int(f[i].max()) < m for i, m in enumerate(mods))


def test_ntt_of_monomials():
    # x^s maps to psi^((2 brv(k)+1) s): a transposed index or wrong sign fails here
    logn, q = 5, W.primes_below(50, 5, 1)[0]
    psi = O.find_psi(q, logn)
    for s in (0, 1, 7, 31):
        a = np.zeros((1, 32), dtype=np.uint64)
        a[0, s] = 1
        got = O.ntt_fwd(a, [q], logn)[0]
        for k in range(32):
            assert int(got[k]) == pow(psi, (2 * pins.brv(k, logn) + 1) * s, q)
