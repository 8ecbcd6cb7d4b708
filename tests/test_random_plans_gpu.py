"""Seeded random parity sweep: workloads (dnum, N, L) and plans (dataflow, chunks,
fused/unfused, radix 4/8/16, caller workspace or the context's) drawn together, so
that combinations the structured tests do not list (odd dnum with ragged digits,
many chunks with radix 16, unfused OutputChunked at two-pass sizes, ...) are checked
bit for bit against the oracle. Keys are uniform residues (the KeySwitch is the same
arithmetic for any key), so the oracle's cost is one KeySwitch per case."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev, first_mismatch, host

pytestmark = pytest.mark.gpu

BASES = (ks.KS_DSOB, ks.KS_DPOB, ks.KS_DSOC, ks.KS_DPOC)
RADIX = (0, ks.KS_RADIX4, ks.KS_RADIX16)


def draw(k: int):
    """Case k: a workload with N in 2^5..2^16 and L+1 up to 48, and a plan."""
    g = W.rng(7000 + k, 15)
    logn = int(g.integers(5, 17))
    L = int(g.integers(0, 48 if logn <= 13 else 24))
    dnum = int(g.integers(1, min(L + 1, 12) + 1))
    base = int(BASES[g.integers(0, 4)])
    v = base | int(RADIX[g.integers(0, 3)]) | (ks.KS_UNFUSED if g.random() < 0.3 else 0)
    chunks = int(g.integers(1, 11)) if base in (ks.KS_DSOC, ks.KS_DPOC) else 0
    own_ws = bool(g.random() < 0.5)
    return (dnum, logn, L), v, chunks, own_ws


@pytest.mark.parametrize("k", range(48))
def test_random_workload_and_plan(k):
    import torch
    cfg, v, chunks, own_ws = draw(k)
    prm = W.make_params(*cfg)
    g = W.rng(8000 + k, 16)
    d = W.uniform_limbs(g, prm.q, prm.N)
    evk = W.uniform_limbs(g, prm.mods * (2 * prm.beta), prm.N).reshape(prm.beta, 2, prm.QP,
                                                                       prm.N)
    want = O.keyswitch(prm, d, evk)
    ctx = ks.Context(prm)
    try:
        ws = None
        if own_ws:
            n = ks.ks_workspace_size(ctx.h, v, chunks)
            ws = torch.empty(n // 8 + 1, dtype=torch.uint64, device="cuda")
        out = ctx.switch(dev(d), dev(evk), variant=v, chunks=chunks, workspace=ws)
        torch.cuda.synchronize()
        got = host(out)
    finally:
        ctx.close()
    name = ks.variant_name(v, chunks)
    assert np.array_equal(got, want), f"{prm.name()} {name}: " + first_mismatch(got, want)


def draw_schedule(k: int):
    """Case k of the schedule sweep: a workload with N in 2^5..2^17 and a plan whose
    stages each take a random radix (or the plan's), each column pass the default or
    the alternative column tile."""
    g = W.rng(11000 + k, 19)
    logn = int(g.integers(5, 18))
    L = int(g.integers(0, 40 if logn <= 13 else (16 if logn <= 16 else 6)))
    dnum = int(g.integers(1, min(L + 1, 10) + 1))
    base = int(BASES[g.integers(0, 4)])
    v = base | int(RADIX[g.integers(0, 3)]) | (ks.KS_UNFUSED if g.random() < 0.25 else 0)
    for st in range(5):
        v |= ks.KS_STAGE_RADIX(st, int(g.integers(0, 4)))
    for bit in (ks.KS_COLALT_INV, ks.KS_COLALT_UPC, ks.KS_COLALT_DNC):
        if g.random() < 0.4:
            v |= bit
    if g.random() < 0.4:
        v |= ks.KS_SPLIT_DOWN
    chunks = int(g.integers(1, 8)) if base in (ks.KS_DSOC, ks.KS_DPOC) else 0
    return (dnum, logn, L), v, chunks


@pytest.mark.parametrize("k", range(32))
def test_random_radix_schedule_and_column_tile(k):
    """Per-stage radix schedules and the alternative column tile (the tuner's search
    space) on random workloads, bit for bit against the oracle."""
    import torch
    cfg, v, chunks = draw_schedule(k)
    prm = W.make_params(*cfg)
    g = W.rng(12000 + k, 20)
    d = W.uniform_limbs(g, prm.q, prm.N)
    evk = W.uniform_limbs(g, prm.mods * (2 * prm.beta), prm.N).reshape(prm.beta, 2, prm.QP,
                                                                       prm.N)
    want = O.keyswitch(prm, d, evk)
    ctx = ks.Context(prm)
    try:
        out = ctx.switch(dev(d), dev(evk), variant=v, chunks=chunks)
        torch.cuda.synchronize()
        got = host(out)
    finally:
        ctx.close()
    name = ks.variant_name(v, chunks)
    assert np.array_equal(got, want), f"{prm.name()} {name}: " + first_mismatch(got, want)


def draw_eval(k: int):
    """Case k of the evaluation sweep: a workload, a level below the top (or the top),
    an operation (KeySwitch, HMUL, HROT with a random Galois element) and a plan."""
    g = W.rng(9000 + k, 17)
    logn = int(g.integers(5, 15))
    L = int(g.integers(1, 40 if logn <= 12 else 20))
    dnum = int(g.integers(1, min(L + 1, 10) + 1))
    level = int(g.integers(0, L + 1))
    op = ("switch", "hmul", "hrot")[int(g.integers(0, 3))]
    base = int(BASES[g.integers(0, 4)])
    v = base | int(RADIX[g.integers(0, 3)]) | (ks.KS_UNFUSED if g.random() < 0.3 else 0)
    chunks = int(g.integers(1, 8)) if base in (ks.KS_DSOC, ks.KS_DPOC) else 0
    rot = 2 * int(g.integers(0, 1 << logn)) + 1  # odd in [1, 2N)
    return (dnum, logn, L), level, op, v, chunks, rot


@pytest.mark.parametrize("k", range(24))
def test_random_level_and_operation(k):
    """KeySwitch, HMUL and HROT at random levels (level views with the top level's key)
    under random plans, against the oracle's level-aware functions."""
    import torch
    cfg, level, op, v, chunks, rot = draw_eval(k)
    prm = W.make_params(*cfg)
    g = W.rng(10000 + k, 18)
    key = W.uniform_limbs(g, prm.mods * (2 * prm.beta), prm.N).reshape(prm.beta, 2, prm.QP,
                                                                       prm.N)
    qs = prm.q[:level + 1]
    x = W.uniform_limbs(g, qs * 2, prm.N).reshape(2, level + 1, prm.N)
    y = W.uniform_limbs(g, qs * 2, prm.N).reshape(2, level + 1, prm.N)
    if op == "switch":
        want = O.keyswitch_level(prm, level, x[1], key)
    elif op == "hmul":
        want = O.hmul(prm, level, x, y, key)
    else:
        want = O.hrot(prm, level, x, rot, key)
    top = ks.Context(prm)
    view = top.at_level(level) if level < prm.L else top
    try:
        kk = dev(key)
        if op == "switch":
            out = view.switch(dev(x[1]), kk, variant=v, chunks=chunks)
        elif op == "hmul":
            out = view.hmul(dev(x), dev(y), kk, variant=v, chunks=chunks)
        else:
            out = view.hrot(dev(x), rot, kk, variant=v, chunks=chunks)
        torch.cuda.synchronize()
        got = host(out)
    finally:
        if view is not top:
            view.close()
        top.close()
    name = ks.variant_name(v, chunks)
    assert np.array_equal(got, want), f"{prm.name()} level {level} {op} {name}: " + \
        first_mismatch(got, want)


@pytest.mark.parametrize("k", range(6))
def test_random_batches(k):
    """Random batches (1-12 jobs, some sharing a context, random plans or KS_AUTO) in
    every batch mode: streams, graph (run twice: capture, then replay), autotuned, and
    the persistent kernel (N >= 2^13); every job's output against the oracle."""
    import torch
    g = W.rng(11000 + k, 19)
    persistent = k % 3 == 2
    njobs = int(g.integers(1, 13))
    cfgs, plans = [], []
    for _ in range(njobs):
        if cfgs and g.random() < 0.3:
            cfgs.append(cfgs[int(g.integers(0, len(cfgs)))])
        else:
            logn = int(g.integers(13 if persistent else 6, 15))
            L = int(g.integers(0, 20))
            cfgs.append((int(g.integers(1, min(L + 1, 8) + 1)), logn, L))
        if g.random() < 0.3:
            plans.append((ks.KS_AUTO, 0))
        else:
            base = int(BASES[g.integers(0, 4)])
            v = base | int(RADIX[g.integers(0, 3)]) | (ks.KS_UNFUSED if g.random() < 0.3 else 0)
            plans.append((v, int(g.integers(1, 6)) if base in (ks.KS_DSOC, ks.KS_DPOC) else 0))
    ctxs, arg, want = {}, [], []
    try:
        for j, cfg in enumerate(cfgs):
            prm = W.make_params(*cfg)
            if cfg not in ctxs:
                ctxs[cfg] = ks.Context(prm)
            gj = W.rng(12000 + 100 * k + j, 20)
            d = W.uniform_limbs(gj, prm.q, prm.N)
            evk = W.uniform_limbs(gj, prm.mods * (2 * prm.beta), prm.N).reshape(
                prm.beta, 2, prm.QP, prm.N)
            out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
            arg.append((ctxs[cfg].h, dev(d), dev(evk), out, *plans[j]))
            want.append(O.keyswitch(prm, d, evk))
        modes = [0, ks.KS_BATCH_GRAPH, ks.KS_BATCH_GRAPH, ks.KS_BATCH_AUTOTUNE]
        if persistent:
            modes += [ks.KS_BATCH_PERSISTENT, ks.KS_BATCH_PERSISTENT | ks.KS_BATCH_GRAPH]
        for flags in modes:
            for a in arg:
                a[3].fill_(3)
            ks.ks_switch_batch(arg, flags)
            if flags & ks.KS_BATCH_PERSISTENT:
                assert ks.ks_batch_status() == ks.KS_OK
            torch.cuda.synchronize()
            for j, a in enumerate(arg):
                got = host(a[3])
                assert np.array_equal(got, want[j]), \
                    f"flags {flags:#x} job {j} {cfgs[j]} {ks.variant_name(*plans[j])}: " + \
                    first_mismatch(got, want[j])
    finally:
        for c in ctxs.values():
            c.close()


def draw_tc(k: int):
    """Case k of the tensor-core sweep: a two-pass workload (N = 2^13..2^17) whose digit
    size alpha is 2..9 (the tensor-core path's range; last digits ragged at random), a
    level (the top, or a view below it), and a plan with KS_BCONV_TC or
    KS_BCONV_TC_DOWN over a random dataflow, chunk count, schedule and split."""
    g = W.rng(13000 + k, 21)
    logn = int(g.integers(13, 18))
    cap = {13: 40, 14: 32, 15: 24, 16: 20, 17: 10}[logn]  # L+1 bound: oracle time
    alpha = int(g.integers(2, 10))
    dnum = int(g.integers(1, max(1, cap // alpha) + 1))
    L = max(alpha, dnum * alpha - int(g.integers(0, alpha))) - 1  # L+1 in (.., dnum*alpha]
    dnum = -(-(L + 1) // alpha)
    level = L if g.random() < 0.7 or L < 1 else int(g.integers(0, L + 1))
    base = int(BASES[g.integers(0, 4)])
    v = base | (ks.KS_BCONV_TC if g.random() < 0.7 else ks.KS_BCONV_TC_DOWN)
    v |= int(RADIX[g.integers(0, 3)])
    for st in range(5):
        if g.random() < 0.5:
            v |= ks.KS_STAGE_RADIX(st, int(g.integers(1, 4)))
    if g.random() < 0.4:
        v |= ks.KS_SPLIT_DOWN
    if g.random() < 0.3:
        v |= ks.KS_COLALT_INV
    chunks = int(g.integers(1, 8)) if base in (ks.KS_DSOC, ks.KS_DPOC) else 0
    return (dnum, logn, L), level, v, chunks


@pytest.mark.parametrize("k", range(24))
def test_random_tensor_core_plans(k):
    """The tensor-core basis conversions under random workloads, levels and plans, bit
    for bit against the oracle."""
    import torch
    cfg, level, v, chunks = draw_tc(k)
    prm = W.make_params(*cfg)
    assert 2 <= prm.alpha <= 9, cfg
    g = W.rng(14000 + k, 22)
    key = W.uniform_limbs(g, prm.mods * (2 * prm.beta), prm.N).reshape(prm.beta, 2, prm.QP,
                                                                       prm.N)
    x = W.uniform_limbs(g, prm.q[:level + 1], prm.N)
    want = O.keyswitch_level(prm, level, x, key)
    top = ks.Context(prm)
    view = top.at_level(level) if level < prm.L else top
    try:
        out = view.switch(dev(x), dev(key), variant=v, chunks=chunks)
        torch.cuda.synchronize()
        got = host(out)
    finally:
        if view is not top:
            view.close()
        top.close()
    name = ks.variant_name(v, chunks)
    assert np.array_equal(got, want), f"{prm.name()} level {level} {name}: " + \
        first_mismatch(got, want)
