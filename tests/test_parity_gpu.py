"""GPU KeySwitch == oracle, bit for bit (integer work: the bar is exact equality).

Covers the single-pass NTT sizes (N <= 4096) and the two-pass ones (N >= 8192),
every dataflow (DSOB, DPOB, DSOC, DPOC) fused and unfused, chunks 1..10 and more
chunks than limbs, ragged last digits and chunks, dnum = 1 and dnum = L+1, the
three plain workloads (2,2^13,7), (2,2^15,10), (4,2^16,35) at full size with
seeds 0-2, key generation, the host-buffer entry point and caller workspaces.
"""
import numpy as np
import pytest

from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev, first_mismatch, host, oracle_case

pytestmark = pytest.mark.gpu

ALL = [(name, v) for name, v in ks.VARIANTS.items()]


def run_gpu(prm, s_from, s_to, a, e, d, variants, chunk_list=(0,)):
    import torch
    ctx = ks.Context(prm)
    try:
        evk = ctx.keygen(dev(s_from), dev(s_to), dev(a), dev(e))
        torch.cuda.synchronize()
        dd = dev(d)
        outs = {}
        for v in variants:
            chunks = chunk_list if v & 0xff in (ks.KS_DSOC, ks.KS_DPOC) else (0,)
            for c in chunks:
                out = ctx.switch(dd, evk, variant=v, chunks=c)
                torch.cuda.synchronize()
                outs[(v, c)] = host(out)
        return host(evk), outs
    finally:
        ctx.close()


def check(cfg, seed, variants, chunk_list=(0,)):
    prm, s_from, s_to, a, e, d, evk_o, out_o = oracle_case(cfg, seed)
    evk_g, outs = run_gpu(prm, s_from, s_to, a, e, d, variants, chunk_list)
    assert np.array_equal(evk_g, evk_o), "keygen: " + first_mismatch(evk_g, evk_o)
    for (v, c), out in outs.items():
        assert np.array_equal(out, out_o), f"variant {v:#x} chunks {c}: " + first_mismatch(
            out, out_o)
        for i, q in enumerate(prm.q):
            assert int(out[:, i].max()) < q


SMALL = [(2, 1, 1), (1, 2, 0), (2, 3, 2), (3, 4, 5), (2, 5, 7), (4, 6, 9), (10, 7, 12),
         (3, 8, 6), (2, 9, 3), (5, 10, 11), (2, 11, 4), (3, 12, 8)]


@pytest.mark.parametrize("cfg", SMALL)
def test_single_pass_sizes_all_variants(cfg):
    vs = [v for _, v in ALL] + [v | ks.KS_UNFUSED for _, v in ALL]
    check(cfg, 1, vs, chunk_list=(1, 2, 3, 7))


TWO_PASS = [(2, 13, 3), (3, 14, 6), (4, 15, 9), (2, 16, 2), (6, 17, 5), (1, 13, 2), (13, 13, 12)]


@pytest.mark.parametrize("cfg", TWO_PASS)
def test_two_pass_sizes_all_variants(cfg):
    vs = [v for _, v in ALL] + [v | ks.KS_UNFUSED for _, v in ALL]
    check(cfg, 2, vs, chunk_list=(2, 5, 64))


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("cfg", [W.C1, W.C2])
def test_plain_workloads_every_variant_and_chunks(cfg, seed):
    vs = [v for _, v in ALL] + [v | ks.KS_UNFUSED for _, v in ALL]
    check(cfg, seed, vs, chunk_list=tuple(range(2, 11)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_c3_every_variant(seed):
    vs = [v for _, v in ALL] + [v | ks.KS_UNFUSED for _, v in ALL]
    chunks = tuple(range(2, 11)) if seed == 0 else (2, 4, 6)
    check(W.C3, seed, vs, chunk_list=chunks)


RADIX_PLANS = [ks.KS_DPOB, ks.KS_DSOB, ks.KS_DPOC]


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("cfg", [W.C2, W.C3])
@pytest.mark.parametrize("radix", [ks.KS_RADIX4, ks.KS_RADIX16])
def test_plain_workloads_radix4_and_radix16(cfg, seed, radix):
    """The radix-4 and radix-16 register rounds (the tuner's other radix schedules) at the
    full (2,2^15,10) and (4,2^16,35) sizes: DPOB, DSOB and DPOC with 2 chunks."""
    check(cfg, seed, [v | radix for v in RADIX_PLANS], chunk_list=(2,))


SCHEDULES = [
    ks.KS_DPOB | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4),
    ks.KS_DPOB | ks.KS_RADIX4 | ks.KS_STAGE_RADIX(ks.KS_ST_UPC, ks.KS_R8)
    | ks.KS_STAGE_RADIX(ks.KS_ST_DNC, ks.KS_R16) | ks.KS_COLTILE_ALT,
    ks.KS_DSOB | ks.KS_STAGE_RADIX(ks.KS_ST_INV, ks.KS_R4)
    | ks.KS_STAGE_RADIX(ks.KS_ST_DNR, ks.KS_R16),
    ks.KS_DPOC | ks.KS_COLTILE_ALT | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R16),
    ks.KS_DPOB | ks.KS_UNFUSED | ks.KS_STAGE_RADIX(ks.KS_ST_UPC, ks.KS_R4) | ks.KS_COLTILE_ALT,
    ks.KS_DPOB | ks.KS_COLALT_INV | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4),
    ks.KS_DSOC | ks.KS_COLALT_UPC | ks.KS_STAGE_RADIX(ks.KS_ST_DNR, ks.KS_R4),
    ks.KS_DPOB | ks.KS_UNFUSED | ks.KS_COLALT_DNC,
    ks.KS_DPOB | ks.KS_SPLIT_DOWN | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4),
    ks.KS_DPOB | ks.KS_RADIX4 | ks.KS_SPLIT_DOWN | ks.KS_STAGE_RADIX(ks.KS_ST_DNR, ks.KS_R8),
    ks.KS_DPOC | ks.KS_SPLIT_DOWN,  # ignored by other plans
]


@pytest.mark.parametrize("cfg", [W.C1, W.C2, W.C3])
def test_plain_workloads_radix_schedules(cfg):
    """Per-stage radix schedules and the alternative column tile at full size."""
    check(cfg, 0, SCHEDULES, chunk_list=(3,))


# the tensor-core plan the benchmark times at (4, 2^16, 35), with and without its split
KM4_TC = ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4) | ks.KS_BCONV_TC


@pytest.mark.parametrize("radix", [0, ks.KS_RADIX4, ks.KS_RADIX16, KM4_TC,
                                   KM4_TC | ks.KS_SPLIT_DOWN])
@pytest.mark.parametrize("cfg", [W.C2, W.C3])
def test_host_entry_points_with_each_radix(cfg, radix):
    """ks_switch_host and ks_switch_host_async (pinned buffers: the input iNTT reads the
    host input over the CPU-GPU link, the last kernel writes the host output) with the
    DPOB plan of each radix and the tensor-core plans, over a ring of three host buffers
    and three calls each."""
    import torch
    prm = W.make_params(*cfg)
    cases = [oracle_case(cfg, seed) for seed in (0, 1, 2)]
    evk_o = cases[0][6]
    ctx = ks.Context(prm)
    try:
        evk = dev(evk_o)
        v = ks.KS_DPOB | radix
        d_hs = [torch.from_numpy(c[5].copy()).pin_memory() for c in cases]
        # one key for the three inputs: seed 0's; the oracle switches the inputs of seeds
        # 1 and 2 under that key
        from oracle import oracle as O
        want = [cases[0][7]] + [O.keyswitch(prm, c[5], evk_o) for c in cases[1:]]
        outs = [torch.full((2, prm.L + 1, prm.N), 3, dtype=torch.uint64).pin_memory()
                for _ in cases]
        for k in range(3):
            ks.ks_switch_host(ctx.h, d_hs[k], evk, outs[k], v, 0)
            assert np.array_equal(outs[k].numpy(), want[k]), f"sync call {k}"
        for o in outs:
            o.fill_(3)
        for k in range(3):
            ks.ks_switch_host_async(ctx.h, d_hs[k], evk, outs[k], v, 0)
        torch.cuda.synchronize()
        for k in range(3):
            assert np.array_equal(outs[k].numpy(), want[k]), f"async call {k}"
    finally:
        ctx.close()


@pytest.mark.parametrize("plan", [ks.KS_DPOB | ks.KS_RADIX4,
                                  ks.KS_DPOB | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4)
                                  | ks.KS_STAGE_RADIX(ks.KS_ST_DNR, ks.KS_R4) | ks.KS_SPLIT_DOWN,
                                  ks.KS_DPOB | KM4_TC, ks.KS_DPOB | KM4_TC | ks.KS_SPLIT_DOWN])
@pytest.mark.parametrize("cfg", [W.C2, W.C3, (2, 12, 5)])
def test_host_async_with_caller_scratch_on_three_streams(cfg, plan):
    """ks_switch_host_async_ws: host-buffer KeySwitches in flight on three streams, each
    with its own scratch (workspace + device copies of the input and result, moved by
    the copy engines), nine calls over a ring of three pinned inputs and nine pinned
    outputs; every result exact, and short scratch or pageable buffers refused."""
    import torch
    prm = W.make_params(*cfg)
    cases = [oracle_case(cfg, seed) for seed in (0, 1, 2)]
    evk_o = cases[0][6]
    from oracle import oracle as O
    want = [cases[0][7]] + [O.keyswitch(prm, c[5], evk_o) for c in cases[1:]]
    ctx = ks.Context(prm)
    try:
        evk = dev(evk_o)
        nbytes = ks.ks_host_workspace_size(ctx.h, plan, 0)
        assert nbytes == ks.ks_workspace_size(ctx.h, plan, 0) + 3 * (prm.L + 1) * prm.N * 8
        streams = [torch.cuda.Stream() for _ in range(3)]
        wss = [torch.empty(nbytes // 8, dtype=torch.uint64, device="cuda") for _ in streams]
        d_hs = [torch.from_numpy(c[5].copy()).pin_memory() for c in cases]
        outs = [torch.full((2, prm.L + 1, prm.N), 3, dtype=torch.uint64).pin_memory()
                for _ in range(9)]
        torch.cuda.synchronize()
        for k in range(9):
            ks.ks_switch_host_async_ws(ctx.h, d_hs[k % 3], evk, outs[k], wss[k % 3], plan, 0,
                                       streams[k % 3])
        torch.cuda.synchronize()
        for k in range(9):
            assert np.array_equal(outs[k].numpy(), want[k % 3]), f"call {k}"
        small = torch.empty(nbytes // 8 - 2, dtype=torch.uint64, device="cuda")
        with pytest.raises(ks.KSError) as ei:
            ks.ks_switch_host_async_ws(ctx.h, d_hs[0], evk, outs[0], small, plan, 0)
        assert ei.value.code == ks.KS_EINVAL
        with pytest.raises(ks.KSError) as ei:  # pageable host memory is refused
            ks.ks_switch_host_async_ws(ctx.h, torch.from_numpy(cases[0][5].copy()), evk,
                                       outs[0], wss[0], plan, 0)
        assert ei.value.code == ks.KS_EINVAL
    finally:
        ctx.close()


def test_host_entry_point_and_workspace():
    import torch
    prm, s_from, s_to, a, e, d, evk_o, out_o = oracle_case(W.C2, 0)
    ctx = ks.Context(prm)
    try:
        evk = dev(evk_o)
        d_h = torch.from_numpy(d.copy()).pin_memory()
        out_h = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64).pin_memory()
        ks.ks_switch_host(ctx.h, d_h, evk, out_h, ks.KS_DPOC, 3)
        assert np.array_equal(out_h.numpy(), out_o)
        for v in (ks.KS_DSOB, ks.KS_DPOC | ks.KS_UNFUSED):
            nbytes = ks.ks_workspace_size(ctx.h, v, 4)
            ws = torch.empty(nbytes // 8, dtype=torch.uint64, device="cuda")
            out = ctx.switch(dev(d), evk, variant=v, chunks=4, workspace=ws)
            assert np.array_equal(host(out), out_o)
            small = torch.empty(nbytes // 8 - 64, dtype=torch.uint64, device="cuda")
            with pytest.raises(ks.KSError) as ei:
                ctx.switch(dev(d), evk, variant=v, chunks=4, workspace=small)
            assert ei.value.code == ks.KS_EINVAL
    finally:
        ctx.close()


def test_bad_calls_return_errors():
    import torch
    prm, s_from, s_to, a, e, d, evk_o, out_o = oracle_case(W.C1, 0)
    ctx = ks.Context(prm)
    try:
        evk = dev(evk_o)
        dd = dev(d)
        out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        lib = ks.load()
        s = torch.cuda.current_stream().cuda_stream
        assert lib.ks_switch(ctx.h, dd.data_ptr() + 8, evk.data_ptr(), out.data_ptr(), 0, 0,
                             None, 0, s) == ks.KS_EALIGN
        assert lib.ks_switch(ctx.h, dd.data_ptr(), evk.data_ptr(), out.data_ptr(), 9, 0, None, 0,
                             s) == ks.KS_EINVAL
        assert lib.ks_switch(ctx.h, dd.data_ptr(), evk.data_ptr(), out.data_ptr(), ks.KS_DSOC,
                             65, None, 0, s) == ks.KS_EINVAL
        # nothing was launched by the failed calls; a good call still works
        ctx.switch(dd, evk, out=out)
        torch.cuda.synchronize()
        assert np.array_equal(host(out), out_o)
        assert ks.ks_sync_status(ctx.h) == ks.KS_OK
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg", [(2, 13, 127), (15, 13, 127)])
def test_maximum_limb_count(cfg):
    """L+1 = 128 ciphertext primes (the library's limit), with 2 and with 15 digits."""
    vs = [ks.KS_DPOB, ks.KS_DSOB, ks.KS_DPOC, ks.KS_DPOB | ks.KS_UNFUSED]
    check(cfg, 0, vs, chunk_list=(3,))


def test_key_multiply_sum_bound_is_enforced():
    """beta * max modulus must stay below 2^64 (one exact 128-bit sum per key multiply):
    19 digits of ~2^60 special primes would overflow and are refused."""
    prm = W.make_params(19, 13, 127)
    assert prm.beta * max(prm.mods) >= 1 << 64
    with pytest.raises(ks.KSError):
        ks.Context(prm)


def test_empty_batch_is_a_no_op():
    ks.ks_switch_batch([], 0)
    ks.ks_switch_batch([], ks.KS_BATCH_GRAPH)
    ks.ks_switch_batch([], ks.KS_BATCH_PERSISTENT)
