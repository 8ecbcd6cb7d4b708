"""HMUL, HROT, their keys, and KeySwitch at lower levels on the GPU, bit for bit
against the oracle (Sec. II-A; Sec. V for switching the dataflow as the level falls)."""
import functools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev, first_mismatch, host

pytestmark = pytest.mark.gpu

PLANS = [(ks.KS_DSOB, 0), (ks.KS_DPOB, 0), (ks.KS_DSOC, 3), (ks.KS_DPOC, 2),
         (ks.KS_DPOB | ks.KS_RADIX4, 0), (ks.KS_DPOB | ks.KS_UNFUSED, 0),
         (ks.KS_DSOC | ks.KS_RADIX16, 2), (ks.KS_DPOC | ks.KS_UNFUSED | ks.KS_RADIX4, 2),
         # the tensor-core conversions (ignored where a context has no tensor-core path)
         (ks.KS_DPOB | ks.KS_BCONV_TC | ks.KS_STAGE_RADIX(ks.KS_ST_KM, ks.KS_R4), 0),
         (ks.KS_DSOC | ks.KS_BCONV_TC_DOWN, 2)]


def rand_ct(prm, level, seed):
    g = W.rng(seed, 7)
    return W.uniform_limbs(g, prm.q[:level + 1] * 2, prm.N).reshape(2, level + 1, prm.N)


@functools.lru_cache(maxsize=8)
def relin_case(cfg, seed):
    prm = W.make_params(*cfg)
    _, s, a, e = W.gen_keys(prm, seed)
    s2 = O.negacyclic_mul_i64(s, s, prm.logn)
    return prm, s, a, e, O.keygen_poly(prm, s2, s, a, e)


@functools.lru_cache(maxsize=8)
def rot_case(cfg, seed, k):
    prm = W.make_params(*cfg)
    _, s, a, e = W.gen_keys(prm, seed)
    sk = O.automorphism_i64(s, prm.logn, k)
    return prm, s, a, e, O.keygen_poly(prm, sk, s, a, e)


@pytest.mark.parametrize("cfg", [(2, 13, 7), (3, 14, 5), (4, 12, 9)])
def test_relin_and_rotation_keys_match_oracle(cfg):
    prm, s, a, e, rlk_o = relin_case(cfg, 1)
    ctx = ks.Context(prm)
    try:
        rlk = ctx.keygen_relin(dev(s), dev(a), dev(e))
        got = host(rlk)
        assert np.array_equal(got, rlk_o), "relin: " + first_mismatch(got, rlk_o)
        for k in (ks.galois_elt(1, prm.N), ks.galois_elt(-3, prm.N), ks.galois_elt(None, prm.N)):
            _, s2, a2, e2, rtk_o = rot_case(cfg, 2, k)
            rtk = ctx.keygen_galois(dev(s2), k, dev(a2), dev(e2))
            got = host(rtk)
            assert np.array_equal(got, rtk_o), f"k={k}: " + first_mismatch(got, rtk_o)
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg", [(2, 13, 7), (3, 15, 9), (2, 11, 4), (4, 16, 12)])
def test_hmul_every_plan(cfg):
    import torch
    prm, s, a, e, rlk_o = relin_case(cfg, 3)
    ct1, ct2 = rand_ct(prm, prm.L, 1), rand_ct(prm, prm.L, 2)
    want = O.hmul(prm, prm.L, ct1, ct2, rlk_o)
    ctx = ks.Context(prm)
    try:
        rlk, c1, c2 = dev(rlk_o), dev(ct1), dev(ct2)
        for v, c in PLANS:
            out = ctx.hmul(c1, c2, rlk, variant=v, chunks=c)
            torch.cuda.synchronize()
            got = host(out)
            assert np.array_equal(got, want), ks.variant_name(v, c) + ": " + \
                first_mismatch(got, want)
        # in place: out aliases ct1
        ctx.hmul(c1, c2, rlk, out=c1)
        torch.cuda.synchronize()
        assert np.array_equal(host(c1), want)
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg,r", [((2, 13, 7), 1), ((3, 14, 5), 5), ((2, 12, 3), None),
                                   ((4, 16, 10), -7)])
def test_hrot_every_plan(cfg, r):
    import torch
    prm = W.make_params(*cfg)
    k = ks.galois_elt(r, prm.N)
    _, s, a, e, rtk_o = rot_case(cfg, 4, k)
    ct = rand_ct(prm, prm.L, 3)
    want = O.hrot(prm, prm.L, ct, k, rtk_o)
    ctx = ks.Context(prm)
    try:
        rtk, c = dev(rtk_o), dev(ct)
        for v, ch in PLANS:
            out = ctx.hrot(c, k, rtk, variant=v, chunks=ch)
            torch.cuda.synchronize()
            got = host(out)
            assert np.array_equal(got, want), ks.variant_name(v, ch) + ": " + \
                first_mismatch(got, want)
        ctx.hrot(c, k, rtk, out=c)  # in place
        torch.cuda.synchronize()
        assert np.array_equal(host(c), want)
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg", [(4, 16, 23), (3, 13, 11), (10, 14, 29)])
def test_level_views_every_plan(cfg):
    """KeySwitch at several levels l < L with the top-level key: every plan bit-exact."""
    import torch
    prm = W.make_params(*cfg)
    s_from, s_to, a, e = W.gen_keys(prm, 5)
    evk_o = O.keygen(prm, s_from, s_to, a, e)
    top = ks.Context(prm)
    try:
        evk = dev(evk_o)
        levels = sorted({prm.L - 1, prm.L - prm.alpha, prm.alpha, prm.alpha - 1, 2, 0})
        for level in levels:
            if level < 0:
                continue
            d = W.uniform_limbs(W.rng(level, 8), prm.q[:level + 1], prm.N)
            want = O.keyswitch_level(prm, level, d, evk_o)
            view = top.at_level(level)
            try:
                assert view.info["top_L"] == prm.L and view.nq == level + 1
                dd = dev(d)
                for v, c in PLANS:
                    out = view.switch(dd, evk, variant=v, chunks=c)
                    torch.cuda.synchronize()
                    got = host(out)
                    assert np.array_equal(got, want), f"level {level} " + \
                        ks.variant_name(v, c) + ": " + first_mismatch(got, want)
            finally:
                view.close()
    finally:
        top.close()


def test_hmul_and_hrot_at_lower_levels():
    import torch
    cfg = (3, 14, 11)
    prm, s, a, e, rlk_o = relin_case(cfg, 6)
    k = ks.galois_elt(2, prm.N)
    _, _, _, _, rtk_o = rot_case(cfg, 6, k)
    top = ks.Context(prm)
    try:
        rlk, rtk = dev(rlk_o), dev(rtk_o)
        for level in (8, 5, 1):
            ct1, ct2 = rand_ct(prm, level, 11), rand_ct(prm, level, 12)
            view = top.at_level(level)
            try:
                got = host(view.hmul(dev(ct1), dev(ct2), rlk))
                want = O.hmul(prm, level, ct1, ct2, rlk_o)
                assert np.array_equal(got, want), f"hmul level {level}: " + \
                    first_mismatch(got, want)
                got = host(view.hrot(dev(ct1), k, rtk))
                torch.cuda.synchronize()
                want = O.hrot(prm, level, ct1, k, rtk_o)
                assert np.array_equal(got, want), f"hrot level {level}: " + \
                    first_mismatch(got, want)
            finally:
                view.close()
    finally:
        top.close()


def test_level_views_in_a_persistent_batch():
    """Level views of different contexts in one persistent launch."""
    import torch
    jobs = []
    ctxs = []
    try:
        for cfg, level, seed in [((4, 16, 23), 13, 0), ((3, 13, 11), 4, 1), ((2, 15, 9), 9, 2),
                                 ((10, 14, 29), 20, 3)]:
            prm = W.make_params(*cfg)
            s_from, s_to, a, e = W.gen_keys(prm, seed)
            evk_o = O.keygen(prm, s_from, s_to, a, e)
            top = ks.Context(prm)
            view = top.at_level(level)
            ctxs += [view, top]
            d = W.uniform_limbs(W.rng(seed, 9), prm.q[:level + 1], prm.N)
            want = O.keyswitch_level(prm, level, d, evk_o)
            out = torch.full((2, level + 1, prm.N), 5, dtype=torch.uint64, device="cuda")
            jobs.append((view, dev(d), dev(evk_o), out, want))
        for flags in (ks.KS_BATCH_PERSISTENT, ks.KS_BATCH_GRAPH):
            ks.ks_switch_batch([(v.h, d, evk, out) for v, d, evk, out, _ in jobs], flags)
            torch.cuda.synchronize()
            for k, (_, _, _, out, want) in enumerate(jobs):
                got = host(out)
                assert np.array_equal(got, want), f"flags {flags} job {k}: " + \
                    first_mismatch(got, want)
    finally:
        for c in ctxs:
            c.close()


def test_eval_argument_checks():
    prm = W.make_params(2, 12, 3)
    ctx = ks.Context(prm)
    try:
        import torch
        ct = torch.zeros((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        rtk = torch.zeros((prm.beta, 2, prm.QP, prm.N), dtype=torch.uint64, device="cuda")
        for bad_k in (0, 2, 2 * prm.N + 1):
            with pytest.raises(ks.KSError):
                ctx.hrot(ct, bad_k, rtk)
        with pytest.raises(ks.KSError):
            ks.ks_context_at_level(ctx.h, prm.L + 1)
        view = ctx.at_level(1)
        try:
            with pytest.raises(ks.KSError):
                ks.ks_context_at_level(view.h, 0)
            s = torch.zeros(prm.N, dtype=torch.int8, device="cuda")
            e = torch.zeros((prm.beta, prm.N), dtype=torch.int32, device="cuda")
            with pytest.raises(ks.KSError):
                view.keygen_relin(s, rtk[:, 0].contiguous(), e)
        finally:
            view.close()
        assert ks.ks_eval_workspace_size(ctx.h, ks.KS_OP_HROT) == \
            ks.ks_eval_workspace_size(ctx.h, ks.KS_OP_SWITCH) + 2 * (prm.L + 1) * prm.N * 8
    finally:
        ctx.close()
