"""Repeated single operations: at single-pass sizes (N <= 2^12) and through the
host-buffer entry point they replay a cached CUDA graph (captured on the second call
with the same plan, buffers and stream); larger sizes launch directly. Every call must
read the buffers' current contents and give the oracle's result."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev, first_mismatch, host, oracle_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [(3, 12, 8), (3, 14, 8)])
@pytest.mark.parametrize("variant,chunks", [(ks.KS_DPOB, 0), (ks.KS_DSOC | ks.KS_RADIX4, 3),
                                            (ks.KS_DSOB | ks.KS_UNFUSED, 0)])
def test_switch_replays_see_new_inputs(cfg, variant, chunks):
    import torch
    cases = [oracle_case(cfg, s) for s in (0, 1, 2)]
    prm = cases[0][0]
    ctx = ks.Context(prm)
    try:
        d = dev(cases[0][5])
        evk = dev(cases[0][6])
        out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        # calls 1 (direct), 2 (capture), 3..6 (replays), inputs changed in place
        for rep in range(6):
            c = cases[rep % 3]
            d.copy_(torch.from_numpy(c[5]).cuda())
            evk.copy_(torch.from_numpy(c[6]).cuda())
            out.fill_(7)
            ctx.switch(d, evk, out, variant=variant, chunks=chunks)
            torch.cuda.synchronize()
            got = host(out)
            assert np.array_equal(got, c[7]), f"call {rep}: " + first_mismatch(got, c[7])
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg", [(2, 12, 5), (2, 13, 5)])
def test_hmul_and_hrot_replays(cfg):
    import torch
    prm = W.make_params(*cfg)
    _, s, a, e = W.gen_keys(prm, 1)
    rlk_o = O.keygen_poly(prm, O.negacyclic_mul_i64(s, s, prm.logn), s, a, e)
    k = ks.galois_elt(3, prm.N)
    rtk_o = O.keygen_poly(prm, O.automorphism_i64(s, prm.logn, k), s, a, e)
    ctx = ks.Context(prm)
    try:
        rlk, rtk = dev(rlk_o), dev(rtk_o)
        ct1 = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        ct2 = torch.empty_like(ct1)
        out = torch.empty_like(ct1)
        for rep in range(5):
            g = W.rng(rep, 12)
            x = W.uniform_limbs(g, prm.q * 2, prm.N).reshape(2, prm.L + 1, prm.N)
            y = W.uniform_limbs(g, prm.q * 2, prm.N).reshape(2, prm.L + 1, prm.N)
            ct1.copy_(torch.from_numpy(x).cuda())
            ct2.copy_(torch.from_numpy(y).cuda())
            ctx.hmul(ct1, ct2, rlk, out)
            torch.cuda.synchronize()
            want = O.hmul(prm, prm.L, x, y, rlk_o)
            assert np.array_equal(host(out), want), f"hmul call {rep}"
            ctx.hrot(ct1, k, rtk, out)
            torch.cuda.synchronize()
            want = O.hrot(prm, prm.L, x, k, rtk_o)
            assert np.array_equal(host(out), want), f"hrot call {rep}"
    finally:
        ctx.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_entry_replays(pinned):
    """ks_switch_host: pinned buffers are captured with their copies into one graph;
    pageable buffers cannot be captured and keep running directly. Every call must
    return the oracle's result for the current contents."""
    import torch
    cfg = (2, 13, 6)
    cases = [oracle_case(cfg, s) for s in (0, 1, 2)]
    prm = cases[0][0]
    ctx = ks.Context(prm)
    try:
        evk = dev(cases[0][6])
        if pinned:
            d_h = torch.empty((prm.L + 1, prm.N), dtype=torch.uint64).pin_memory()
            out_h = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64).pin_memory()
        else:
            d_h = np.empty((prm.L + 1, prm.N), dtype=np.uint64)
            out_h = np.empty((2, prm.L + 1, prm.N), dtype=np.uint64)
        for rep in range(5):
            c = cases[rep % 3]
            evk.copy_(torch.from_numpy(c[6]).cuda())
            if pinned:
                d_h.copy_(torch.from_numpy(c[5]))
            else:
                d_h[...] = c[5]
            ks.ks_switch_host(ctx.h, d_h, evk, out_h)
            got = out_h.numpy() if pinned else out_h
            assert np.array_equal(got, c[7]), f"call {rep}: " + first_mismatch(got, c[7])
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg", [(2, 12, 5), (2, 13, 6), (2, 15, 4)])
def test_host_async_queue(cfg):
    """ks_switch_host_async: several host-buffer KeySwitches queued on one stream with a
    ring of pinned inputs and outputs (single-pass graph replay at 2^12, chained direct
    launches above), synchronized once; every output is the oracle's for its input.
    Pageable buffers are refused."""
    import torch
    cases = [oracle_case(cfg, s) for s in (0, 1, 2)]
    prm = cases[0][0]
    ctx = ks.Context(prm)
    try:
        evks = [dev(c[6]) for c in cases]
        d_hs = [torch.from_numpy(c[5]).pin_memory() for c in cases]
        out_hs = [torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64).pin_memory()
                  for _ in range(6)]
        for rep in range(6):
            out_hs[rep].fill_(0)
            ks.ks_switch_host_async(ctx.h, d_hs[rep % 3], evks[rep % 3], out_hs[rep])
        torch.cuda.synchronize()
        for rep in range(6):
            got, want = out_hs[rep].numpy(), cases[rep % 3][7]
            assert np.array_equal(got, want), f"call {rep}: " + first_mismatch(got, want)
        d_pageable = np.array(cases[0][5])
        with pytest.raises(ks.KSError):
            ks.ks_switch_host_async(ctx.h, d_pageable, evks[0], out_hs[0])
        # pinned but 8 bytes off a 16-byte boundary: refused before any launch
        big = torch.empty(d_hs[0].numel() + 1, dtype=torch.uint64).pin_memory()
        d_off = big[1:].view(prm.L + 1, prm.N)
        assert d_off.data_ptr() % 16 == 8
        with pytest.raises(ks.KSError) as err:
            ks.ks_switch_host_async(ctx.h, d_off, evks[0], out_hs[0])
        assert err.value.code == ks.KS_EALIGN
    finally:
        ctx.close()
