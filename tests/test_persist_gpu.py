"""The persistent batch kernel (one launch for a whole uneven batch) on the GPU.

Outputs are compared bit for bit with the oracle's KeySwitch of each job; the
bounded-wait test makes one stage dependency unreachable and checks that the
kernel gives up, reports KS_ETIMEOUT and leaves the context usable."""
import time

import numpy as np
import pytest

from paper_2603_16692_gb300 import ks
from tests.gpu_util import dev, first_mismatch, host, oracle_case

pytestmark = pytest.mark.gpu


def _jobs(cfgs, seeds):
    import torch
    ctxs, jobs = {}, []
    for cfg, seed in zip(cfgs, seeds):
        prm, s_from, s_to, a, e, d, evk_o, out_o = oracle_case(cfg, seed)
        if cfg not in ctxs:
            ctxs[cfg] = ks.Context(prm)
        out = torch.full((2, prm.L + 1, prm.N), 3, dtype=torch.uint64, device="cuda")
        jobs.append((ctxs[cfg], dev(d), dev(evk_o), out, out_o))
    return ctxs, jobs


CFGS = [(2, 13, 7), (3, 14, 9), (2, 13, 7), (5, 15, 12), (4, 16, 6), (3, 14, 9), (7, 17, 8),
        (10, 13, 20), (2, 17, 5), (6, 16, 30)]
SEEDS = [0, 1, 2, 0, 1, 4, 0, 3, 5, 6]


def _check(jobs, tag):
    for k, (_, _, _, out, want) in enumerate(jobs):
        got = host(out)
        assert np.array_equal(got, want), f"{tag} job {k} {CFGS[k]}: " + first_mismatch(got, want)


@pytest.mark.parametrize("graph", [False, True])
def test_persistent_batch_matches_oracle(graph):
    import torch
    ctxs, jobs = _jobs(CFGS, SEEDS)
    flags = ks.KS_BATCH_PERSISTENT | (ks.KS_BATCH_GRAPH if graph else 0)
    try:
        arg = [(c.h, d, evk, out) for c, d, evk, out, _ in jobs]
        for rep in range(3):  # with a graph: capture, then replays
            for _, _, _, out, _ in jobs:
                out.fill_(3)
            ks.ks_switch_batch(arg, flags)
            assert ks.ks_batch_status() == ks.KS_OK
            torch.cuda.synchronize()
            _check(jobs, f"rep {rep}")
    finally:
        for c in ctxs.values():
            c.close()


def test_persistent_single_job_every_size():
    import torch
    for cfg in [(2, 13, 3), (3, 14, 5), (2, 15, 4), (4, 16, 7), (3, 17, 2)]:
        ctxs, jobs = _jobs([cfg], [7])
        try:
            c, d, evk, out, want = jobs[0]
            ks.ks_switch_batch([(c.h, d, evk, out)], ks.KS_BATCH_PERSISTENT)
            assert ks.ks_batch_status() == ks.KS_OK
            torch.cuda.synchronize()
            got = host(out)
            assert np.array_equal(got, want), f"{cfg}: " + first_mismatch(got, want)
        finally:
            for c in ctxs.values():
                c.close()


def test_persistent_rejects_unsupported_sizes():
    ctxs, jobs = _jobs([(2, 12, 4)], [0])
    try:
        c, d, evk, out, _ = jobs[0]
        with pytest.raises(ks.KSError):
            ks.ks_switch_batch([(c.h, d, evk, out)], ks.KS_BATCH_PERSISTENT)
        with pytest.raises(ks.KSError):
            ks.ks_switch_batch([(c.h, d, evk, out)], ks.KS_BATCH_TEST_STALL)
    finally:
        for c in ctxs.values():
            c.close()


def test_persistent_bounded_wait_times_out_and_recovers():
    """A dependency that never completes: the wait gives up after its limit (about
    2 s of device time), the status is KS_ETIMEOUT, and the next batch is correct."""
    import torch
    cfgs, seeds = CFGS[:4], SEEDS[:4]
    ctxs, jobs = _jobs(cfgs, seeds)
    try:
        arg = [(c.h, d, evk, out) for c, d, evk, out, _ in jobs]
        t0 = time.monotonic()
        ks.ks_switch_batch(arg, ks.KS_BATCH_PERSISTENT | ks.KS_BATCH_TEST_STALL)
        assert ks.ks_batch_status() == ks.KS_ETIMEOUT
        assert time.monotonic() - t0 < 30
        # the context still works
        for _, _, _, out, _ in jobs:
            out.fill_(3)
        ks.ks_switch_batch(arg, ks.KS_BATCH_PERSISTENT)
        assert ks.ks_batch_status() == ks.KS_OK
        torch.cuda.synchronize()
        for k, (_, _, _, out, want) in enumerate(jobs):
            got = host(out)
            assert np.array_equal(got, want), f"job {k}: " + first_mismatch(got, want)
    finally:
        for c in ctxs.values():
            c.close()
