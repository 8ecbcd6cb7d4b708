"""Independent mathematical references used to pin the oracle (Python ints only).

Nothing here reuses the oracle's code: these are the textbook definitions
(direct polynomial evaluation, schoolbook negacyclic convolution, Chinese
remaindering) written out in exact integer arithmetic.
"""
from __future__ import annotations

import numpy as np


def brv(k: int, bits: int) -> int:
    r = 0
    for _ in range(bits):
        r = (r << 1) | (k & 1)
        k >>= 1
    return r


def ntt_direct(a, q: int, psi: int, logn: int):
    """a_hat[k] = sum_n a[n] psi^((2 brv(k)+1) n) mod q  (O(N^2))."""
    n = 1 << logn
    out = []
    for k in range(n):
        w = pow(psi, 2 * brv(k, logn) + 1, q)
        s, wn = 0, 1
        for c in a:
            s = (s + int(c) * wn) % q
            wn = wn * w % q
        out.append(s)
    return out


def negacyclic_mul(a, b, q: int):
    """Schoolbook product in Z_q[x]/(x^N + 1)."""
    n = len(a)
    out = [0] * n
    for i in range(n):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] = (out[k] + ai * int(b[j])) % q
            else:
                out[k - n] = (out[k - n] - ai * int(b[j])) % q
    return out


def crt(residues, mods) -> int:
    """The unique x in [0, prod mods) with x = r_i mod m_i (textbook CRT)."""
    M = 1
    for m in mods:
        M *= m
    x = 0
    for r, m in zip(residues, mods):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M


def prod(xs) -> int:
    r = 1
    for x in xs:
        r *= int(x)
    return r


def centred(x: int, m: int) -> int:
    x %= m
    return x - m if x > m // 2 else x


def to_residues(v, m: int) -> np.ndarray:
    """Signed ints -> canonical residues mod m (uint64)."""
    return np.array([int(x) % m for x in np.asarray(v).ravel()], dtype=np.uint64).reshape(
        np.shape(v))
