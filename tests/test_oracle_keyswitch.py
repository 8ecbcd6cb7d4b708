"""Pins of the oracle's basis conversion, ModDown, key multiply and full KeySwitch.

Sec. II-A fixes the step order (iNTT -> BConv -> NTT, key multiply, then
iNTT -> BConv -> NTT back to level l) and that BConv is only "approximately
equivalent". The checks below pin each step with exact big-integer
arithmetic: the CRT value of the converted limbs, floor division by P, the
a = e = 0 special case, and the decryption-noise bound.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16692_gb300 import workload as W
from tests import pins


def _rand_limbs(g, mods, n):
    return np.stack([g.integers(0, m, size=n, dtype=np.uint64) for m in mods])


@pytest.mark.parametrize("ns,nd,logn", [(1, 3, 4), (3, 5, 5), (6, 11, 6), (9, 12, 3)])
def test_bconv_is_crt_plus_small_multiple(ns, nd, logn):
    g = np.random.default_rng(ns * 100 + nd)
    src = W.primes_below(50, logn, ns + nd)[:ns]
    dst = list(W.primes_below(50, logn, ns + nd)[ns:])
    dst[-1] = W.primes_below(60, logn, 1)[0]
    x = _rand_limbs(g, src, 1 << logn)
    y = O.bconv(x, src, dst, logn)
    S = pins.prod(src)
    for n in range(1 << logn):
        xv = pins.crt([x[i, n] for i in range(ns)], src)
        # y = X mod m_t with X = x + u*S, 0 <= u < ns, the same u for every target
        u = (int(y[0, n]) - xv) * pow(S, -1, dst[0]) % dst[0]
        assert 0 <= u < ns
        X = xv + u * S
        for t, m in enumerate(dst):
            assert int(y[t, n]) == X % m


def test_bconv_exact_when_value_small():
    # x < S/ns keeps the fast conversion exact for a single source (u = 0)
    logn = 4
    src = W.primes_below(50, logn, 1)
    dst = W.primes_below(60, logn, 3)
    x = np.arange(16, dtype=np.uint64).reshape(1, 16) * np.uint64(12345)
    y = O.bconv(x, src, dst, logn)
    for t, m in enumerate(dst):
        assert [int(v) for v in y[t]] == [int(v) % m for v in x[0]]


@pytest.mark.parametrize("cfg", [(2, 4, 3), (3, 5, 5), (2, 6, 7), (4, 4, 8)])
def test_moddown_is_floor_division_by_P(cfg):
    prm = W.make_params(*cfg)
    g = np.random.default_rng(sum(cfg))
    acc = _rand_limbs(g, prm.mods, prm.N)
    out = O.moddown(prm, acc)
    xc = O.ntt_inv(acc, prm.mods, prm.logn)       # coefficient form over Q u P
    yc = O.ntt_inv(out, prm.q, prm.logn)          # coefficient form over Q
    P = pins.prod(prm.p)
    Q = pins.prod(prm.q)
    for n in range(prm.N):
        x = pins.crt(xc[:, n], prm.mods)
        y = pins.crt(yc[:, n], prm.q)
        u = (x // P - y) % Q
        assert 0 <= u < prm.alpha


def test_moddown_of_multiple_of_P_is_exact():
    prm = W.make_params(2, 6, 7)
    g = np.random.default_rng(5)
    yh = _rand_limbs(g, prm.q, prm.N)             # NTT form, mod Q
    acc = np.zeros((prm.QP, prm.N), dtype=np.uint64)
    for i, q in enumerate(prm.q):
        Pq = pins.prod(prm.p) % q
        acc[i] = [int(v) * Pq % q for v in yh[i]]
    # P * y = 0 mod every p_k
    assert np.array_equal(O.moddown(prm, acc), yh)


def _keys(prm, seed, zero_noise=False):
    s_from, s_to, a, e = W.gen_keys(prm, seed)
    if zero_noise:
        a = np.zeros_like(a)
        e = np.zeros_like(e)
    return s_from, s_to, a, e


def _ntt_small(v, prm):
    return O.ntt_fwd(np.stack([pins.to_residues(v, m) for m in prm.q]), prm.q, prm.logn)


@pytest.mark.parametrize("cfg", [(2, 4, 3), (3, 5, 6), (2, 6, 7), (4, 5, 9), (10, 4, 12)])
def test_keyswitch_zero_noise_key_gives_exact_product(cfg):
    """With a = e = 0 the key is (P g_j s_from, 0): the switched pair is exactly (d*s_from, 0)."""
    prm = W.make_params(*cfg)
    s_from, s_to, a, e = _keys(prm, 1, zero_noise=True)
    evk = O.keygen(prm, s_from, s_to, a, e)
    d = W.gen_input(prm, 3)
    out = O.keyswitch(prm, d, evk)
    assert not out[1].any()
    dc = O.ntt_inv(d, prm.q, prm.logn)
    for i, q in enumerate(prm.q):
        want = pins.negacyclic_mul(dc[i], pins.to_residues(s_from, q), q)
        got = O.ntt_inv(out[0][i:i + 1], [q], prm.logn)[0]
        assert [int(v) for v in got] == want


def noise_bound(prm) -> int:
    """|E| <= alpha (N+1) + ceil(19 beta N alpha Q_D,max / P) for the floor ModDown:
    key-multiply error sum_j X_j e_j / P with |X_j| < |D_j| Q_Dj, |e| <= 19, plus the
    dropped [acc]_P / P (<= N+1) and the BConv overflow u (<= (alpha-1)(N+1))."""
    P = pins.prod(prm.p)
    qd = max(pins.prod([prm.q[i] for i in prm.digit(j)]) for j in range(prm.beta))
    return prm.alpha * (prm.N + 1) + -(-(19 * prm.beta * prm.N * prm.alpha * qd) // P)


def decrypt_error(prm, d, out, s_from, s_to):
    """E = out0 + out1*s_to - d*s_from over Q, centred per prime; asserts all primes agree."""
    sf, st = _ntt_small(s_from, prm), _ntt_small(s_to, prm)
    e_hat = np.zeros_like(d)
    for i, q in enumerate(prm.q):
        o0 = out[0][i].astype(object)
        o1 = out[1][i].astype(object)
        e_hat[i] = ((o0 + o1 * st[i].astype(object) - d[i].astype(object) * sf[i].astype(object))
                    % q).astype(np.uint64)
    ec = O.ntt_inv(e_hat, prm.q, prm.logn)
    cen = np.array([[pins.centred(int(v), q) for v in ec[i]] for i, q in enumerate(prm.q)],
                   dtype=np.int64)
    assert (cen == cen[0]).all(), "error polynomial differs across primes"
    return cen[0]


@pytest.mark.parametrize("cfg", [(2, 5, 3), (3, 6, 8), (2, 8, 7), (4, 7, 11)])
def test_keyswitch_noise_within_bound_small(cfg):
    prm = W.make_params(*cfg)
    s_from, s_to, a, e = _keys(prm, 2)
    evk = O.keygen(prm, s_from, s_to, a, e)
    d = W.gen_input(prm, 4)
    out = O.keyswitch(prm, d, evk)
    E = decrypt_error(prm, d, out, s_from, s_to)
    assert np.abs(E).max() <= noise_bound(prm)
    assert np.abs(E).max() > 0


def test_keyswitch_noise_within_bound_c1():
    prm = W.make_params(*W.C1)
    s_from, s_to, a, e = _keys(prm, 0)
    evk = O.keygen(prm, s_from, s_to, a, e)
    d = W.gen_input(prm, 0)
    out = O.keyswitch(prm, d, evk)
    E = decrypt_error(prm, d, out, s_from, s_to)
    B = noise_bound(prm)
    assert np.abs(E).max() <= B
    # expected size O(alpha sqrt N): far below the worst case
    assert np.abs(E).max() < 20 * prm.alpha * math.sqrt(prm.N)


def test_keyswitch_trace_structure():
    """ext_j equals d on the digit's own limbs; acc is the digit sum of ext * evk."""
    prm = W.make_params(3, 5, 7)
    s_from, s_to, a, e = _keys(prm, 3)
    evk = O.keygen(prm, s_from, s_to, a, e)
    d = W.gen_input(prm, 5)
    out, ext, acc = O.keyswitch(prm, d, evk, trace=True)
    for j in range(prm.beta):
        for i in prm.digit(j):
            assert np.array_equal(ext[j, i], d[i])
    # ModUp of digit j is a BConv of the iNTT of its limbs, then NTT
    dc = O.ntt_inv(d, prm.q, prm.logn)
    j = 1
    dig = list(prm.digit(j))
    others = [t for t in range(prm.QP) if t not in dig]
    y = O.bconv(dc[dig], [prm.q[i] for i in dig], [prm.mods[t] for t in others], prm.logn)
    yh = O.ntt_fwd(y, [prm.mods[t] for t in others], prm.logn)
    assert np.array_equal(ext[j, others], yh)
    for c in range(2):
        for t in (0, prm.QP - 1):
            m = prm.mods[t]
            want = sum(ext[jj, t].astype(object) * evk[jj, c, t].astype(object)
                       for jj in range(prm.beta)) % m
            assert np.array_equal(acc[c, t], want.astype(np.uint64))
    assert np.array_equal(O.moddown(prm, acc[0]), out[0])


def test_keygen_relation():
    """b_j + a_j s_to - e_j is P*s_from on the digit's Q-limbs and 0 on every other limb."""
    prm = W.make_params(2, 5, 5)
    s_from, s_to, a, e = _keys(prm, 4)
    evk = O.keygen(prm, s_from, s_to, a, e)
    P = pins.prod(prm.p)
    for j in range(prm.beta):
        for t, m in enumerate(prm.mods):
            sc = O.ntt_inv(evk[j, 0, t:t + 1], [m], prm.logn)[0]
            ac = O.ntt_inv(evk[j, 1, t:t + 1], [m], prm.logn)[0]
            lhs = [(int(b) + x - int(ee)) % m for b, x, ee in
                   zip(sc, pins.negacyclic_mul(ac, pins.to_residues(s_to, m), m), e[j])]
            g = P % m if (t < prm.L + 1 and t in prm.digit(j)) else 0
            want = [g * int(v) % m for v in pins.to_residues(s_from, m)]
            assert lhs == want
