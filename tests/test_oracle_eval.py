"""Pins of the oracle's HMUL, HROT and KeySwitch at lower levels (Sec. II-A, Sec. V).

HMUL = tensor product + KeySwitch of the degree-2 part under s^2; HROT = Galois
automorphism + KeySwitch under sigma_k(s); a KeySwitch at level l < L uses the
top level's key restricted to the remaining primes. Each is pinned by exact
identities (direct evaluation at the roots of x^N + 1, schoolbook products, a
key made from scratch on the smaller basis, exact zero special cases) and by the
decryption-noise bound of the KeySwitch.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16692_gb300 import workload as W
from tests import pins


@dataclasses.dataclass
class LevelParams:
    """The (q, p, alpha) of a KeySwitch at level l with the top level's alpha."""
    logn: int
    L: int
    q: tuple
    p: tuple
    alpha: int

    @property
    def N(self):
        return 1 << self.logn

    @property
    def beta(self):
        return -(-(self.L + 1) // self.alpha)

    def digit(self, j):
        return range(j * self.alpha, min((j + 1) * self.alpha, self.L + 1))


def level_params(prm, level):
    return LevelParams(prm.logn, level, prm.q[:level + 1], prm.p, prm.alpha)


def noise_bound(lp) -> int:
    """Same bound as the top-level KeySwitch, over the level's digits."""
    P = pins.prod(lp.p)
    qd = max(pins.prod([lp.q[i] for i in lp.digit(j)]) for j in range(lp.beta))
    return lp.alpha * (lp.N + 1) + -(-(19 * lp.beta * lp.N * lp.alpha * qd) // P)


def ntt_of_int_poly(v, mods, logn):
    return O.ntt_fwd(np.stack([pins.to_residues(v, m) for m in mods]), mods, logn)


def error_poly(lp, out, want_hat, s_to):
    """E = out0 + out1*s_to - want over Q_l (all NTT form), centred per prime, checked to
    agree across the primes."""
    st = ntt_of_int_poly(s_to, lp.q, lp.logn)
    e_hat = np.zeros((len(lp.q), lp.N), dtype=np.uint64)
    for i, q in enumerate(lp.q):
        v = (out[0][i].astype(object) + out[1][i].astype(object) * st[i].astype(object)
             - want_hat[i].astype(object)) % q
        e_hat[i] = v.astype(np.uint64)
    ec = O.ntt_inv(e_hat, lp.q, lp.logn)
    cen = np.array([[pins.centred(int(v), q) for v in ec[i]] for i, q in enumerate(lp.q)],
                   dtype=np.int64)
    assert (cen == cen[0]).all(), "error polynomial differs across primes"
    return cen[0]


def rand_ct(g, mods, n, count=2):
    return np.stack([np.stack([g.integers(0, m, size=n, dtype=np.uint64) for m in mods])
                     for _ in range(count)])


def mulmod_hat(x, y, mods):
    return np.stack([(x[i].astype(object) * y[i].astype(object) % m).astype(np.uint64)
                     for i, m in enumerate(mods)])


def addmod_hat(x, y, mods):
    return np.stack([((x[i].astype(object) + y[i].astype(object)) % m).astype(np.uint64)
                     for i, m in enumerate(mods)])


# ---------------------------------------------------------------- small-integer helpers

@pytest.mark.parametrize("logn", [1, 3, 5])
def test_negacyclic_mul_i64_is_schoolbook(logn):
    g = np.random.default_rng(logn)
    a = g.integers(-5, 6, size=1 << logn)
    b = g.integers(-5, 6, size=1 << logn)
    got = O.negacyclic_mul_i64(a, b, logn)
    q = 1000003
    want = pins.negacyclic_mul([int(v) % q for v in a], [int(v) % q for v in b], q)
    assert [int(v) % q for v in got] == want
    # x^(N-1) * x = x^N = -1
    e1 = np.zeros(1 << logn, dtype=np.int64)
    e1[-1] = 1
    x = np.zeros(1 << logn, dtype=np.int64)
    x[1 % (1 << logn)] = 1
    if logn > 0:
        prod = O.negacyclic_mul_i64(e1, x, logn)
        assert prod[0] == -1 and not prod[1:].any()


@pytest.mark.parametrize("logn,k", [(3, 5), (4, 3), (5, 31), (6, 127), (4, 1)])
def test_automorphism_is_substitution_at_the_roots(logn, k):
    """sigma_k(a)(w) = a(w^k) at every root w = psi^(2j+1) of x^N + 1 (direct evaluation)."""
    N = 1 << logn
    q = W.primes_below(50, logn, 1)[0]
    psi = O.find_psi(q, logn)
    g = np.random.default_rng(k)
    a = g.integers(-20, 21, size=N)
    s = O.automorphism_i64(a, logn, k)

    def ev(poly, w):
        acc, wn = 0, 1
        for c in poly:
            acc = (acc + int(c) * wn) % q
            wn = wn * w % q
        return acc

    for j in range(N):
        w = pow(psi, 2 * j + 1, q)
        assert ev(s, w) == ev(a, pow(w, k, q))


@pytest.mark.parametrize("logn", [3, 6])
def test_automorphism_group_laws(logn):
    N = 1 << logn
    g = np.random.default_rng(logn + 7)
    a = g.integers(-9, 10, size=N)
    b = g.integers(-9, 10, size=N)
    k = pow(5, 3, 2 * N)
    kinv = pow(k, -1, 2 * N)
    assert np.array_equal(O.automorphism_i64(O.automorphism_i64(a, logn, k), logn, kinv), a)
    assert np.array_equal(O.automorphism_i64(a, logn, 1), a)
    # a ring homomorphism: sigma(a b) = sigma(a) sigma(b)
    lhs = O.automorphism_i64(O.negacyclic_mul_i64(a, b, logn), logn, k)
    rhs = O.negacyclic_mul_i64(O.automorphism_i64(a, logn, k), O.automorphism_i64(b, logn, k),
                               logn)
    assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("logn,k", [(4, 5), (5, 2 * 32 - 1), (6, 25)])
def test_automorph_ntt_slots(logn, k):
    """The NTT-form automorphism: slot j of the result is a(w_j^k), w_j = psi^(2 brv(j)+1)."""
    N = 1 << logn
    mods = W.primes_below(50, logn, 2)
    g = np.random.default_rng(logn)
    ah = np.stack([g.integers(0, m, size=N, dtype=np.uint64) for m in mods])
    got = O.automorph_ntt(ah, mods, logn, k)
    ac = O.ntt_inv(ah, mods, logn)
    for c, q in enumerate(mods):
        psi = O.find_psi(q, logn)
        for j in range(N):
            w = pow(psi, 2 * pins.brv(j, logn) + 1, q)
            wk = pow(w, k, q)
            acc, wn = 0, 1
            for v in ac[c]:
                acc = (acc + int(v) * wn) % q
                wn = wn * wk % q
            assert int(got[c, j]) == acc


# ---------------------------------------------------------------- keys

def test_keygen_poly_equals_keygen_for_ternary_keys():
    prm = W.make_params(3, 5, 7)
    s_from, s_to, a, e = W.gen_keys(prm, 1)
    assert np.array_equal(O.keygen_poly(prm, s_from.astype(np.int64), s_to, a, e),
                          O.keygen(prm, s_from, s_to, a, e))


def test_keygen_poly_relation_for_s_squared():
    """b_j + a_j s - e_j = [P g_j] s^2 on every limb, with s^2 from the schoolbook product."""
    prm = W.make_params(2, 4, 3)
    _, s, a, e = W.gen_keys(prm, 2)
    s2 = O.negacyclic_mul_i64(s, s, prm.logn)
    evk = O.keygen_poly(prm, s2, s, a, e)
    P = pins.prod(prm.p)
    for j in range(prm.beta):
        for t, m in enumerate(prm.mods):
            bc = O.ntt_inv(evk[j, 0, t:t + 1], [m], prm.logn)[0]
            ac = O.ntt_inv(evk[j, 1, t:t + 1], [m], prm.logn)[0]
            lhs = [(int(b) + x - int(ee)) % m for b, x, ee in
                   zip(bc, pins.negacyclic_mul(ac, pins.to_residues(s, m), m), e[j])]
            gj = P % m if (t <= prm.L and t in prm.digit(j)) else 0
            assert lhs == [gj * (int(v) % m) % m for v in s2]


# ---------------------------------------------------------------- KeySwitch at level l

def _restricted_key_randomness(prm, level, a, e):
    """The top key's randomness on the limbs of level `level`: rows q_0..q_l, then P."""
    lp = level_params(prm, level)
    rows = list(range(level + 1)) + [prm.L + 1 + k for k in range(prm.alpha)]
    return a[:lp.beta][:, rows], e[:lp.beta]


@pytest.mark.parametrize("cfg,level", [((2, 5, 9), 8), ((3, 4, 8), 5), ((4, 5, 11), 8),
                                       ((2, 4, 5), 2), ((3, 5, 8), 8)])
def test_level_keyswitch_equals_fresh_small_basis(cfg, level):
    """KS at level l with the top key == KS at the top of the basis q_0..q_l, P with a key
    made there from the same randomness (the top key restricted to the remaining limbs)."""
    prm = W.make_params(*cfg)
    s_from, s_to, a, e = W.gen_keys(prm, 3)
    evk = O.keygen(prm, s_from, s_to, a, e)
    lp = level_params(prm, level)
    dn = -(-(level + 1) // prm.alpha)
    small = W.Params(dn, prm.logn, level, prm.q[:level + 1], prm.p)
    assert small.alpha == prm.alpha and small.beta == lp.beta
    a_l, e_l = _restricted_key_randomness(prm, level, a, e)
    evk_small = O.keygen(small, s_from, s_to, a_l, e_l)
    d = W.gen_input(small, 4)
    assert np.array_equal(O.keyswitch_level(prm, level, d, evk), O.keyswitch(small, d, evk_small))
    if level == prm.L:
        assert np.array_equal(O.keyswitch_level(prm, level, d, evk), O.keyswitch(prm, d, evk))


@pytest.mark.parametrize("cfg", [(2, 6, 7), (3, 5, 10)])
def test_level_keyswitch_noise_within_bound(cfg):
    prm = W.make_params(*cfg)
    s_from, s_to, a, e = W.gen_keys(prm, 5)
    evk = O.keygen(prm, s_from, s_to, a, e)
    for level in (0, prm.alpha - 1, prm.alpha, prm.L - 1):
        lp = level_params(prm, level)
        g = np.random.default_rng(level)
        d = rand_ct(g, lp.q, lp.N, 1)[0]
        out = O.keyswitch_level(prm, level, d, evk)
        want = mulmod_hat(d, ntt_of_int_poly(s_from, lp.q, lp.logn), lp.q)
        E = error_poly(lp, out, want, s_to)
        assert np.abs(E).max() <= noise_bound(lp)


# ---------------------------------------------------------------- HMUL

def _relin_key(prm, seed):
    _, s, a, e = W.gen_keys(prm, seed)
    s2 = O.negacyclic_mul_i64(s, s, prm.logn)
    return s, O.keygen_poly(prm, s2, s, a, e)


def test_hmul_with_zero_degree_one_part_is_the_exact_product():
    """x1 = 0: the KeySwitch input x1 y1 is 0, so out = (x0 y0, x0 y1) exactly."""
    prm = W.make_params(2, 5, 5)
    _, rlk = _relin_key(prm, 1)
    g = np.random.default_rng(3)
    ct1 = rand_ct(g, prm.q, prm.N)
    ct1[1] = 0
    ct2 = rand_ct(g, prm.q, prm.N)
    out = O.hmul(prm, prm.L, ct1, ct2, rlk)
    assert np.array_equal(out[0], mulmod_hat(ct1[0], ct2[0], prm.q))
    assert np.array_equal(out[1], mulmod_hat(ct1[0], ct2[1], prm.q))


@pytest.mark.parametrize("cfg,level", [((2, 5, 5), 5), ((3, 6, 8), 4), ((2, 7, 3), 3)])
def test_hmul_decrypts_to_the_product(cfg, level):
    """out0 + out1 s = (x0 + x1 s)(y0 + y1 s) + E with E within the KeySwitch bound."""
    prm = W.make_params(*cfg)
    s, rlk = _relin_key(prm, 2)
    lp = level_params(prm, level)
    g = np.random.default_rng(sum(cfg))
    ct1 = rand_ct(g, lp.q, lp.N)
    ct2 = rand_ct(g, lp.q, lp.N)
    out = O.hmul(prm, level, ct1, ct2, rlk)
    sh = ntt_of_int_poly(s, lp.q, lp.logn)
    m1 = addmod_hat(ct1[0], mulmod_hat(ct1[1], sh, lp.q), lp.q)
    m2 = addmod_hat(ct2[0], mulmod_hat(ct2[1], sh, lp.q), lp.q)
    E = error_poly(lp, out, mulmod_hat(m1, m2, lp.q), s)
    assert np.abs(E).max() <= noise_bound(lp)


# ---------------------------------------------------------------- HROT

def _rot_key(prm, seed, k):
    _, s, a, e = W.gen_keys(prm, seed)
    sk = O.automorphism_i64(s, prm.logn, k)
    return s, O.keygen_poly(prm, sk, s, a, e)


@pytest.mark.parametrize("cfg,level,r", [((2, 5, 5), 5, 1), ((3, 6, 8), 6, 3), ((2, 6, 7), 2, -1)])
def test_hrot_decrypts_to_the_rotation(cfg, level, r):
    """out0 + out1 s = sigma_k(c0 + c1 s) + E (k = 5^r mod 2N; r = -1: conjugation)."""
    prm = W.make_params(*cfg)
    k = 2 * prm.N - 1 if r < 0 else pow(5, r, 2 * prm.N)
    s, rtk = _rot_key(prm, 4, k)
    lp = level_params(prm, level)
    g = np.random.default_rng(level + r)
    ct = rand_ct(g, lp.q, lp.N)
    out = O.hrot(prm, level, ct, k, rtk)
    sh = ntt_of_int_poly(s, lp.q, lp.logn)
    m = addmod_hat(ct[0], mulmod_hat(ct[1], sh, lp.q), lp.q)
    want = O.automorph_ntt(m, lp.q, lp.logn, k)
    E = error_poly(lp, out, want, s)
    assert np.abs(E).max() <= noise_bound(lp)


def test_hrot_identity_element_keeps_c0():
    """k = 1 with a = e = 0 (key (P g_j s, 0)): out = (c0 + c1 s, 0) exactly."""
    prm = W.make_params(2, 5, 5)
    _, s, a, e = W.gen_keys(prm, 6)
    rtk = O.keygen_poly(prm, s.astype(np.int64), s, np.zeros_like(a), np.zeros_like(e))
    g = np.random.default_rng(9)
    ct = rand_ct(g, prm.q, prm.N)
    out = O.hrot(prm, prm.L, ct, 1, rtk)
    sh = ntt_of_int_poly(s, prm.q, prm.logn)
    assert np.array_equal(out[0], addmod_hat(ct[0], mulmod_hat(ct[1], sh, prm.q), prm.q))
    assert not out[1].any()
