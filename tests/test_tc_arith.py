"""The arithmetic behind the tensor-core basis conversion, checked on the CPU.

The kernel (paper_2603_16692_gb300/csrc/ks_tc.cu) computes S = sum_i x_i c_i exactly
from bf16 bytes and fp32 sums: v_s = sum_i sum_{a+b=s} x_ia c_ib (+ 2^23), then the
32-bit word arithmetic of its recombination. These tests emulate that in numpy float32
(in random summation orders) and in wrapped 32/64-bit integers, up to the largest
source count the path accepts (15) and with all-ones bytes (the worst case of the bound
v_s < 2^23), and compare with Python's exact integers.
"""
import numpy as np
import pytest

M32, M64 = (1 << 32) - 1, (1 << 64) - 1
E = 0x4B000000


def byte_sums_f32(xs, cs, rng):
    """fp32 accumulators of the MMA: 2^23 + the byte products of slot s, summed in a
    random order (the tensor core's order is unspecified)."""
    terms = [[] for _ in range(16)]
    for x, c in zip(xs, cs):
        for a in range(8):
            for b in range(8):
                terms[a + b].append(np.float32(((x >> (8 * a)) & 255) * ((c >> (8 * b)) & 255)))
    out = []
    for s in range(16):
        t = np.array(terms[s] + [np.float32(2 ** 23)], dtype=np.float32)
        rng.shuffle(t)
        acc = np.float32(0)
        for v in t:
            acc = np.float32(acc + v)
        out.append(acc)
    return out


def recombine(bits):
    """The kernel's tc_sum on the fp32 bit patterns (wrapped integer arithmetic)."""
    P = [((bits[2 * k] + ((bits[2 * k + 1] << 8) & M32) - E) & M32) for k in range(7)]
    P.append((bits[14] - E) & M32)
    Q = [(P[2 * m] + (P[2 * m + 1] << 16)) & M64 for m in range(4)]
    lo = (Q[0] + ((Q[1] << 32) & M64)) & M64
    hi = ((Q[1] >> 32) + Q[2] + ((Q[3] << 32) & M64) + (1 if lo < Q[0] else 0)) & M64
    return lo | (hi << 64)


@pytest.mark.parametrize("ns", [1, 2, 9, 15])
@pytest.mark.parametrize("kind", ["random", "max"])
def test_byte_split_sums_are_exact(ns, kind):
    rng = np.random.default_rng(ns * 7 + len(kind))
    for _ in range(3):
        if kind == "max":
            xs = [(1 << 62) - 1] * ns
            cs = [(1 << 62) - 1] * ns
        else:
            xs = [int(rng.integers(0, 1 << 62, dtype=np.uint64)) for _ in range(ns)]
            cs = [int(rng.integers(0, 1 << 62, dtype=np.uint64)) for _ in range(ns)]
        sums = byte_sums_f32(xs, cs, rng)
        bits = [int(np.float32(v).view(np.uint32)) for v in sums]
        for s, v in enumerate(sums):
            exact = 2 ** 23 + sum(((x >> (8 * a)) & 255) * ((c >> (8 * (s - a))) & 255)
                                  for x, c in zip(xs, cs) for a in range(8) if 0 <= s - a <= 7)
            assert exact < 2 ** 24 and float(v) == exact, (s, float(v), exact)
            assert bits[s] == E + exact - 2 ** 23
        assert recombine(bits) == sum(x * c for x, c in zip(xs, cs))


def test_sixteen_sources_is_the_bound():
    """16 all-ones sources keep every slot below 2^23 (the bf16 1.0 x 2^23 row then stays
    exact), 17 would not; the path takes at most 15 sources plus that row."""
    assert 16 * 8 * 255 * 255 < 2 ** 23 <= 17 * 8 * 255 * 255
