"""Bit-exact parity at the two remaining workload configurations: the 64-job uneven
batch (every job checked, in every batch mode) and the selector sweep's parameter range
(its largest point, (10, 2^17, 60), and a seeded sample of the others).

Keys are uniform residues here (the KeySwitch is the same arithmetic for any key; key
generation itself is checked against the oracle elsewhere), so the oracle's cost is one
KeySwitch per job."""
import functools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev, first_mismatch, host

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def job_case(cfg, seed):
    prm = W.make_params(*cfg)
    g = W.rng(seed, 13)
    d = W.uniform_limbs(g, prm.q, prm.N)
    evk = W.uniform_limbs(g, prm.mods * (2 * prm.beta), prm.N).reshape(prm.beta, 2, prm.QP,
                                                                       prm.N)
    return prm, d, evk, O.keyswitch(prm, d, evk)


def test_batch64_every_job_every_mode():
    import torch
    jobs = W.batch_jobs(0)
    assert len(jobs) == 64
    ctxs, arg, want = {}, [], []
    try:
        for k, cfg in enumerate(jobs):
            prm, d, evk, out_o = job_case(cfg, 1000 + k)
            if cfg not in ctxs:
                ctxs[cfg] = ks.Context(prm)
            out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
            arg.append((ctxs[cfg].h, dev(d), dev(evk), out))
            want.append(out_o)
        for flags in (0, ks.KS_BATCH_GRAPH | ks.KS_BATCH_AUTOTUNE, ks.KS_BATCH_PERSISTENT,
                      ks.KS_BATCH_PERSISTENT | ks.KS_BATCH_GRAPH):
            for _, _, _, out in arg:
                out.fill_(9)
            ks.ks_switch_batch(arg, flags)
            if flags & ks.KS_BATCH_PERSISTENT:
                assert ks.ks_batch_status() == ks.KS_OK
            torch.cuda.synchronize()
            for k, (_, _, _, out) in enumerate(arg):
                got = host(out)
                assert np.array_equal(got, want[k]), f"flags {flags:#x} job {k} {jobs[k]}: " + \
                    first_mismatch(got, want[k])
    finally:
        for c in ctxs.values():
            c.close()


def sweep_sample():
    pts = W.selector_points(0, 200)
    g = W.rng(7, 14)
    pick = sorted(g.choice(np.arange(1, 200), size=8, replace=False).tolist())
    return [pts[0]] + [pts[i] for i in pick]


@pytest.mark.parametrize("cfg", sweep_sample())
def test_sweep_points_selector_candidates(cfg):
    """The four plans the selector chooses among, on sweep points (the largest first)."""
    import torch
    prm, d, evk, out_o = job_case(tuple(cfg), 2000)
    ctx = ks.Context(prm)
    try:
        dd, ee = dev(d), dev(evk)
        for v, c in ((ks.KS_DPOB, 0), (ks.KS_DSOB, 0), (ks.KS_DPOB | ks.KS_RADIX4, 0),
                     (ks.KS_DPOC, 2)):
            out = ctx.switch(dd, ee, variant=v, chunks=c)
            torch.cuda.synchronize()
            got = host(out)
            assert np.array_equal(got, out_o), ks.variant_name(v, c) + ": " + \
                first_mismatch(got, out_o)
    finally:
        ctx.close()
