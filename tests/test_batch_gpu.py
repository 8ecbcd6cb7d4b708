"""Batched KeySwitch (ks_switch_batch), the radix-4 kernels and the tuner, on the GPU.

Every output is compared bit for bit with the oracle's KeySwitch of the same job."""
import numpy as np
import pytest

from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev, first_mismatch, host, oracle_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("radix", [4, 16])
@pytest.mark.parametrize("cfg", [(2, 5, 3), (3, 11, 7), (2, 13, 5), (4, 15, 9), (6, 16, 11),
                                 (3, 17, 4), (4, 14, 8)])
def test_radix4_and_16_every_variant(cfg, radix):
    import torch
    prm, s_from, s_to, a, e, d, evk_o, out_o = oracle_case(cfg, 3)
    ctx = ks.Context(prm)
    try:
        evk, dd = dev(evk_o), dev(d)
        rf = ks.KS_RADIX4 if radix == 4 else ks.KS_RADIX16
        for v in (ks.KS_DSOB, ks.KS_DPOB, ks.KS_DSOC, ks.KS_DPOC):
            for fu in (0, ks.KS_UNFUSED):
                for c in ((0,) if v in (ks.KS_DSOB, ks.KS_DPOB) else (2, 3)):
                    out = ctx.switch(dd, evk, variant=v | rf | fu, chunks=c)
                    torch.cuda.synchronize()
                    got = host(out)
                    assert np.array_equal(got, out_o), f"{ks.variant_name(v | rf | fu, c)}: " + \
                        first_mismatch(got, out_o)
    finally:
        ctx.close()


def _jobs(cfgs, seeds):
    """[(ctx, d, evk, out, want)] with contexts shared between equal configs."""
    import torch
    ctxs, jobs = {}, []
    for cfg, seed in zip(cfgs, seeds):
        prm, s_from, s_to, a, e, d, evk_o, out_o = oracle_case(cfg, seed)
        if cfg not in ctxs:
            ctxs[cfg] = ks.Context(prm)
        out = torch.full((2, prm.L + 1, prm.N), 3, dtype=torch.uint64, device="cuda")
        jobs.append((ctxs[cfg], dev(d), dev(evk_o), out, out_o))
    return ctxs, jobs


@pytest.mark.parametrize("flags", [0, ks.KS_BATCH_GRAPH, ks.KS_BATCH_AUTOTUNE,
                                   ks.KS_BATCH_GRAPH | ks.KS_BATCH_AUTOTUNE])
def test_batch_uneven_jobs(flags):
    import torch
    cfgs = [(2, 13, 7), (3, 14, 9), (2, 13, 7), (5, 15, 12), (2, 13, 7), (4, 16, 6),
            (3, 14, 9), (2, 12, 4), (7, 17, 8)]
    seeds = [0, 1, 2, 0, 3, 1, 4, 2, 0]
    ctxs, jobs = _jobs(cfgs, seeds)
    try:
        arg = [(c.h, d, evk, out) for c, d, evk, out, _ in jobs]
        for rep in range(2):  # second call replays the captured graph
            for _, _, _, out, _ in jobs:
                out.fill_(3)
            ks.ks_switch_batch(arg, flags)
            torch.cuda.synchronize()
            for k, (_, _, _, out, want) in enumerate(jobs):
                got = host(out)
                assert np.array_equal(got, want), f"rep {rep} job {k} {cfgs[k]}: " + \
                    first_mismatch(got, want)
    finally:
        for c in ctxs.values():
            c.close()


def test_batch_graph_replay_sees_new_inputs():
    """A replayed graph reads the buffers' current contents."""
    import torch
    cfg = (2, 14, 6)
    prm0, *_, d0, evk0, out0 = oracle_case(cfg, 0)
    prm1, *_, d1, evk1, out1 = oracle_case(cfg, 1)
    ctx = ks.Context(prm0)
    try:
        d = dev(d0)
        evk = dev(evk0)
        outs = [torch.empty((2, prm0.L + 1, prm0.N), dtype=torch.uint64, device="cuda")
                for _ in range(20)]
        arg = [(ctx.h, d, evk, o) for o in outs]
        ks.ks_switch_batch(arg, ks.KS_BATCH_GRAPH)
        torch.cuda.synchronize()
        assert all(np.array_equal(host(o), out0) for o in outs)
        # same pointers, new contents: key of seed 1 with input of seed 1
        d.copy_(dev(d1))
        evk.copy_(dev(evk1))
        ks.ks_switch_batch(arg, ks.KS_BATCH_GRAPH)
        torch.cuda.synchronize()
        assert all(np.array_equal(host(o), out1) for o in outs)
    finally:
        ctx.close()


def test_tuner_picks_a_valid_plan_and_writes_result():
    import torch
    prm, s_from, s_to, a, e, d, evk_o, out_o = oracle_case(W.C2, 0)
    ctx = ks.Context(prm)
    try:
        out = torch.zeros((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        v, c = ks.ks_tune(ctx.h, dev(d), dev(evk_o), out, 1)
        assert v & 0xff in (ks.KS_DSOB, ks.KS_DPOB, ks.KS_DSOC, ks.KS_DPOC)
        assert np.array_equal(host(out), out_o)
        out2 = ctx.switch(dev(d), dev(evk_o))  # KS_AUTO now uses the tuned plan
        torch.cuda.synchronize()
        assert np.array_equal(host(out2), out_o)
    finally:
        ctx.close()


SPLIT = ks.KS_DPOB | ks.KS_SPLIT_DOWN


@pytest.mark.parametrize("flags", [0, ks.KS_BATCH_GRAPH])
def test_batch_split_moddown_plans(flags):
    """Jobs naming the split-ModDown plan (second stream per context) in a batch, plain
    and captured into a graph (two groups of one context fork onto the same side
    stream), replayed twice, bit for bit against the oracle."""
    import torch
    cfgs = [(2, 13, 7), (4, 16, 9), (2, 13, 7), (3, 15, 6), (4, 16, 9)]
    seeds = [0, 1, 2, 3, 4]
    plans = [SPLIT, SPLIT | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4), ks.KS_DPOB, SPLIT,
             SPLIT | ks.KS_RADIX4]
    ctxs, jobs = _jobs(cfgs, seeds)
    try:
        arg = [(c.h, d, evk, out, v, 0) for (c, d, evk, out, _), v in zip(jobs, plans)]
        for rep in range(2):
            for _, _, _, out, _ in jobs:
                out.fill_(3)
            ks.ks_switch_batch(arg, flags)
            torch.cuda.synchronize()
            for k, (_, _, _, out, want) in enumerate(jobs):
                got = host(out)
                assert np.array_equal(got, want), f"rep {rep} job {k} {cfgs[k]}: " + \
                    first_mismatch(got, want)
    finally:
        for c in ctxs.values():
            c.close()


def test_split_moddown_from_two_streams_on_one_context():
    """Two caller streams (own workspaces) switching on one context with the split plan:
    the context's fork / join is serialized per call, every result exact."""
    import torch
    cfg = (4, 16, 11)
    cases = [oracle_case(cfg, s) for s in (0, 1)]
    prm = cases[0][0]
    ctx = ks.Context(prm)
    try:
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        n = ks.ks_workspace_size(ctx.h, SPLIT, 0) // 8 + 1
        wss = [torch.empty(n, dtype=torch.uint64, device="cuda") for _ in streams]
        ins = [(dev(c[5]), dev(c[6])) for c in cases]
        outs = [torch.full((2, prm.L + 1, prm.N), 3, dtype=torch.uint64, device="cuda")
                for _ in streams]
        torch.cuda.synchronize()
        for rep in range(6):
            q = rep % 2
            with torch.cuda.stream(streams[q]):
                ctx.switch(ins[q][0], ins[q][1], outs[q], SPLIT, 0, wss[q], streams[q])
        torch.cuda.synchronize()
        for q in range(2):
            assert np.array_equal(host(outs[q]), cases[q][7]), f"stream {q}"
    finally:
        ctx.close()
