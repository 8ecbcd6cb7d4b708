"""Measurement entry points: the per-kernel profile's operation counts (split into
128-bit multiply-accumulate terms and Shoup products) and the arithmetic calibration
kernels that give the measured ceiling for the integer-bound kernels."""
import math

import pytest

from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import workload as W
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def test_calibration_rates_are_finite_and_plausible():
    bf = ks.ks_calibrate(ks.KS_CAL_BUTTERFLY, 2048)
    mac = ks.ks_calibrate(ks.KS_CAL_MAC, 512)
    for r in (bf, mac):
        assert math.isfinite(r) and 1e10 < r < 1e14, (bf, mac)


def test_calibration_rejects_bad_arguments():
    for kind, iters in ((0, 16), (3, 16), (ks.KS_CAL_MAC, 0)):
        with pytest.raises(ks.KSError):
            ks.ks_calibrate(kind, iters)


def test_profile_counts_key_multiply_terms():
    """DigitParallel/OutputBulk at (2, 2^15, 10): the fused ModUp-row/key-multiply launch
    does 2 * beta * (L+1+alpha) key-multiply terms per coefficient plus one ModUp term
    per own limb (L+1), all 128-bit accumulations; its butterflies are the rest. Its
    achieved rate stays within the measured ceiling of that arithmetic."""
    import torch
    prm = W.make_params(2, 15, 10)
    ctx = ks.Context(prm)
    try:
        s_from, s_to, a, e = (dev(x) for x in W.gen_keys(prm, 0))
        evk = ctx.keygen(s_from, s_to, a, e)
        d = dev(W.gen_input(prm, 0))
        out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        for _ in range(3):
            ctx.switch(d, evk, out, variant=ks.KS_DPOB)
        torch.cuda.synchronize()
        ks.ks_profile_begin()
        reps = 20
        for _ in range(reps):
            ctx.switch(d, evk, out, variant=ks.KS_DPOB)
        stats = {s["name"]: s for s in ks.ks_profile_end()}
    finally:
        ctx.close()
    km = stats["modup_row_keymult"]
    assert km["launches"] == reps
    qp = prm.L + 1 + prm.alpha
    want = (2 * prm.beta * qp + prm.L + 1) * prm.N
    assert km["macs"] / reps == want
    assert km["ops"] > km["macs"]
    for name in ("intt_row(d)", "intt_col(d)", "intt_row(accP)", "intt_col(accP)"):
        assert stats[name]["macs"] == 0 and stats[name]["ops"] > 0
    for s in stats.values():
        assert 0 <= s["macs"] <= s["ops"]
    bf = ks.ks_calibrate(ks.KS_CAL_BUTTERFLY, 8192)
    mac = ks.ks_calibrate(ks.KS_CAL_MAC, 2048)
    t_ceil = km["macs"] / mac + (km["ops"] - km["macs"]) / bf
    assert t_ceil / (km["ms"] / 1e3) <= 1.5, (t_ceil, km["ms"])


def test_profile_counts_tensor_core_conversions():
    """With KS_BCONV_TC at (4, 2^16, 35) the two column conversions count their products
    as tensor-core FLOPs (tc_ap * 256 per target point, alpha = 9 -> tc_ap = 10, each
    digit's targets in pairs) and only one REDC per output as a MAC term; the integer
    plan's launches count no tensor FLOPs."""
    import torch
    prm = W.make_params(*W.C3)
    ctx = ks.Context(prm)
    try:
        s_from, s_to, a, e = (dev(x) for x in W.gen_keys(prm, 0))
        evk = ctx.keygen(s_from, s_to, a, e)
        d = dev(W.gen_input(prm, 0))
        out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
        got = {}
        for v in (ks.KS_DPOB | ks.KS_BCONV_TC, ks.KS_DPOB):
            ctx.switch(d, evk, out, variant=v)
            torch.cuda.synchronize()
            ks.ks_profile_begin()
            ctx.switch(d, evk, out, variant=v)
            got[v] = {s["name"]: s for s in ks.ks_profile_end()}
    finally:
        ctx.close()
    nq, qp, N = prm.L + 1, prm.L + 1 + prm.alpha, prm.N
    assert prm.alpha == 9
    tc = got[ks.KS_DPOB | ks.KS_BCONV_TC]
    up_targets = prm.beta * qp - nq  # every digit converts onto the limbs it lacks
    up_padded = sum((qp - min(nq, (j + 1) * prm.alpha) + j * prm.alpha + 1) // 2 * 2
                    for j in range(prm.beta))
    assert tc["modup_col"]["macs"] == up_targets * N
    assert tc["modup_col"]["tensor_flops"] == up_padded * N * 10 * 256
    assert tc["moddown_col"]["macs"] == 2 * nq * N
    assert tc["moddown_col"]["tensor_flops"] == 2 * ((nq + 1) // 2 * 2) * N * 10 * 256
    for s in got[ks.KS_DPOB].values():
        assert s["tensor_flops"] == 0
    for name in ("modup_row_keymult", "moddown_row"):
        assert tc[name]["tensor_flops"] == 0
