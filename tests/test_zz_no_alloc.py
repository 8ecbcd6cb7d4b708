"""ks_switch_noalloc, the entry point for callers that cannot allocate device memory
when they switch keys (a fixed allocator or memory-pool budget, or a real-time
integration that must not call the allocator after start-up): its scratch is a
static device array in the library. Its output must equal ks_switch's on two calls
in a row (the second call sees the first call's leftover scratch), at every size,
including the single-pass sizes N <= 2^12 for which ks_switch replays cached graphs.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("cfg,variant,chunks", [(W.C2, ks.KS_DPOB, 0), (W.C3, ks.KS_DSOC, 4),
                                                (W.C1, ks.KS_DPOC | ks.KS_UNFUSED, 3),
                                                ((2, 12, 5), ks.KS_DPOB, 0),
                                                ((3, 11, 8), ks.KS_DSOC, 2)])
def test_noalloc_equals_ks_switch_two_calls(cfg, variant, chunks):
    import torch
    prm = W.make_params(*cfg)
    ctx = ks.Context(prm)
    try:
        s_from, s_to, a, e = W.gen_keys(prm, 7)
        evk = ctx.keygen(_dev(s_from), _dev(s_to), _dev(a), _dev(e))
        lib = ks.load()
        stream = torch.cuda.current_stream().cuda_stream
        # the same output buffer on both calls (a repeated call with the same buffers
        # is the case ks_switch hands to its graph cache at N <= 2^12)
        got = torch.full((2, prm.L + 1, prm.N), 7, dtype=torch.uint64, device="cuda")
        d = torch.empty((prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        for call, seed in enumerate((11, 12)):
            d.copy_(_dev(W.gen_input(prm, seed)))
            want = ctx.switch(d, evk, variant=variant, chunks=chunks)
            got.fill_(7)
            rc = lib.ks_switch_noalloc(ctx.h, d.data_ptr(), evk.data_ptr(), got.data_ptr(),
                                       variant, chunks, stream)
            assert rc == ks.KS_OK, ks.strerror(rc)
            torch.cuda.synchronize()
            assert torch.equal(got, want), f"call {call}: differs from ks_switch"
    finally:
        ctx.close()


def test_noalloc_rejects_workloads_beyond_the_static_scratch():
    import torch
    prm = W.make_params(*W.C3)
    ctx = ks.Context(prm)
    try:
        need = ks.ks_workspace_size(ctx.h, ks.KS_DPOB, 0)
        assert need > ks.ks_noalloc_scratch_bytes()
        d = torch.zeros((prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        evk = torch.zeros((prm.beta, 2, prm.QP, prm.N), dtype=torch.uint64, device="cuda")
        out = torch.full((2, prm.L + 1, prm.N), 5, dtype=torch.uint64, device="cuda")
        rc = ks.load().ks_switch_noalloc(ctx.h, d.data_ptr(), evk.data_ptr(), out.data_ptr(),
                                         ks.KS_DPOB, 0, torch.cuda.current_stream().cuda_stream)
        assert rc == ks.KS_EINVAL
        torch.cuda.synchronize()
        assert bool((out == 5).all()), "a rejected call must not launch anything"
        with pytest.raises(ValueError):
            ks.ks_switch_noalloc(ctx.h, d, evk, out, ks.KS_DPOB, 0)
    finally:
        ctx.close()
