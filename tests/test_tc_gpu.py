"""Tensor-core basis conversions (KS_BCONV_TC) == oracle, bit for bit.

The ModUp / ModDown BConv on tcgen05 (byte-split bf16 operands, fp32 sums, exact
128-bit recombination, one REDC) must give the same words as the integer path and the
oracle: every dataflow and chunk count, ragged last digits, dnum = 1, the three plain
workloads at full size with seeds 0-2, alpha up to 9 (the path's limit), with the split
ModDown and radix schedules, in batches and on the host-buffer and allocation-free
entry points. Contexts outside the path's range (alpha = 1 or > 9, single-pass N)
ignore the flag.
"""
import numpy as np
import pytest

from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev, first_mismatch, host, oracle_case
from tests.test_parity_gpu import check

pytestmark = pytest.mark.gpu

TC = ks.KS_BCONV_TC
BASES = [ks.KS_DPOB, ks.KS_DSOB, ks.KS_DPOC, ks.KS_DSOC]


@pytest.mark.parametrize("cfg", [(2, 13, 3), (3, 14, 6), (4, 15, 9), (2, 16, 2), (1, 13, 2),
                                 (6, 17, 5), (13, 13, 12), (3, 12, 8)])
def test_tc_two_pass_sizes_every_dataflow(cfg):
    """Small two-pass shapes (alpha 1..3; alpha = 1 and N = 2^12 ignore the flag),
    chunk counts 2, 5 and more chunks than limbs."""
    check(cfg, 2, [v | TC for v in BASES], chunk_list=(2, 5, 64))


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("cfg", [W.C1, W.C2, W.C3])
def test_tc_plain_workloads(cfg, seed):
    chunks = (2, 3, 7) if cfg != W.C3 or seed == 0 else (2,)
    check(cfg, seed, [v | TC for v in BASES], chunk_list=chunks)


@pytest.mark.parametrize("cfg", [(2, 14, 17), (4, 16, 33), (7, 17, 60), (2, 14, 20)])
def test_tc_alpha_limits(cfg):
    """alpha = 9 (the most K slots, 10) with two full digits, with a ragged last digit,
    at 2^17 with seven digits, and alpha = 11 (beyond the path: the flag is ignored)."""
    check(cfg, 1, [ks.KS_DPOB | TC, ks.KS_DSOC | TC], chunk_list=(3,))


TC_SCHEDULES = [
    ks.KS_DPOB | TC | ks.KS_SPLIT_DOWN | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4)
    | ks.KS_STAGE_RADIX(ks.KS_ST_DNR, ks.KS_R4),
    ks.KS_DPOB | TC | ks.KS_RADIX4 | ks.KS_COLALT_INV,
    ks.KS_DPOB | TC | ks.KS_RADIX16 | ks.KS_SPLIT_DOWN,
    ks.KS_DSOB | TC | ks.KS_STAGE_RADIX(ks.KS_ST_INV, ks.KS_R16),
    ks.KS_DPOB | TC | ks.KS_UNFUSED,  # unfused plans ignore the flag
]


@pytest.mark.parametrize("cfg", [W.C2, W.C3, (10, 17, 60)])
def test_tc_with_schedules(cfg):
    check(cfg, 0, TC_SCHEDULES, chunk_list=(2,))


def test_tc_flag_reported_by_context_info():
    for cfg, want in [(W.C3, 1), (W.C2, 1), ((6, 17, 5), 0), ((3, 12, 8), 0),
                      ((2, 16, 17), 1), ((2, 16, 19), 0)]:
        ctx = ks.Context(W.make_params(*cfg))
        try:
            assert ks.ks_context_info(ctx.h)["tc"] == want, cfg
        finally:
            ctx.close()


def test_tc_batch_and_entry_points():
    """Three jobs in one batch launch (grid z), the host-buffer entry point and the
    allocation-free one, all with the TC plan, against the oracle."""
    import torch
    cfg = W.C2
    prm = W.make_params(*cfg)
    cases = [oracle_case(cfg, s) for s in (0, 1, 2)]
    ctx = ks.Context(prm)
    try:
        v = ks.KS_DPOB | TC | ks.KS_SPLIT_DOWN
        evks, ds, outs = [], [], []
        for (_, s_from, s_to, a, e, d, _, _) in cases:
            evks.append(ctx.keygen(dev(s_from), dev(s_to), dev(a), dev(e)))
            ds.append(dev(d))
            outs.append(torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda"))
        jobs = [(ctx.h, ds[k], evks[k], outs[k], v, 0) for k in range(3)]
        for flags in (0, ks.KS_BATCH_GRAPH):
            for o in outs:
                o.fill_(3)
            ks.ks_switch_batch(jobs, flags)
            torch.cuda.synchronize()
            for k in range(3):
                got, want = host(outs[k]), cases[k][7]
                assert np.array_equal(got, want), f"batch {flags} job {k}: " + \
                    first_mismatch(got, want)
        # host buffers (pinned) through the synchronous host entry point
        d_h = torch.from_numpy(cases[1][5]).pin_memory()
        out_h = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64).pin_memory()
        ks.ks_switch_host(ctx.h, d_h, evks[1], out_h, v, 0)
        assert np.array_equal(out_h.numpy(), cases[1][7]), "host entry point"
        # allocation-free entry point
        got = torch.full((2, prm.L + 1, prm.N), 9, dtype=torch.uint64, device="cuda")
        ks.ks_switch_noalloc(ctx.h, ds[2], evks[2], got, v, 0)
        torch.cuda.synchronize()
        assert np.array_equal(host(got), cases[2][7]), "noalloc entry point"
    finally:
        ctx.close()


TCD = ks.KS_BCONV_TC_DOWN
TCD_PLANS = [
    ks.KS_DPOB | TCD,
    ks.KS_DSOB | TCD,
    ks.KS_DPOC | TCD,
    ks.KS_DPOB | TCD | ks.KS_SPLIT_DOWN | ks.KS_STAGE_RADIX(ks.KS_ST_UPC, ks.KS_R16)
    | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4) | ks.KS_COLALT_UPC,
    ks.KS_DPOB | TCD | TC | ks.KS_RADIX4,  # both flags: both conversions
    ks.KS_DPOB | TCD | ks.KS_UNFUSED,  # unfused plans ignore the flag
]


@pytest.mark.parametrize("cfg", [W.C2, W.C3, (10, 17, 60), (2, 14, 17)])
def test_tc_down_only(cfg):
    """KS_BCONV_TC_DOWN: the ModDown conversion on the tensor cores, the ModUp one on the
    integer path (its own radix and column tile), every dataflow."""
    check(cfg, 2, TCD_PLANS, chunk_list=(3,))
