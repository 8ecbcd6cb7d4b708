"""Shared set-up for the GPU parity tests: seeded inputs, oracle results (cached), and
the CUDA path driven through the C-ABI binding."""
from __future__ import annotations

import functools

import numpy as np

from oracle import oracle as O
from paper_2603_16692_gb300 import workload as W


@functools.lru_cache(maxsize=16)
def oracle_case(cfg: tuple, seed: int):
    """(prm, s_from, s_to, a, e, d, evk, out) with evk and out from the oracle."""
    prm = W.make_params(*cfg)
    s_from, s_to, a, e = W.gen_keys(prm, seed)
    d = W.gen_input(prm, seed)
    evk = O.keygen(prm, s_from, s_to, a, e)
    out = O.keyswitch(prm, d, evk)
    return prm, s_from, s_to, a, e, d, evk, out


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy()


def first_mismatch(got: np.ndarray, want: np.ndarray) -> str:
    bad = np.argwhere(got != want)
    if len(bad) == 0:
        return "equal"
    idx = tuple(bad[0])
    return f"{len(bad)} mismatches, first at {idx}: got {got[idx]} want {want[idx]}"
