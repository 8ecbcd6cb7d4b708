"""The selector MLP on the GPU: forward pass and gradients of the library's CUDA
kernels against the float64 CPU oracle, training, and the regret the trained
network gains over the methods without it (best fixed dataflow, the paper's
footprint rule), on the held-out points of the committed GB300 sweep."""
import os

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2603_16692_gb300 import ks
from paper_2603_16692_gb300 import selector as S
from paper_2603_16692_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _case(seed, b):
    g = np.random.default_rng(seed)
    p = (g.normal(0, 0.3, size=M.NP)).astype(np.float32)
    x = g.normal(0, 1, size=(b, 6)).astype(np.float32)
    t = g.normal(0, 1, size=(b, 4)).astype(np.float32)
    mask = (g.random((b, 4)) < 0.9).astype(np.float32)
    return p, x, t, mask


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("b", [1, 7, 160, 256, 257, 700])
def test_mlp_forward_and_gradient_match_oracle(b):
    import torch
    p, x, t, mask = _case(b, b)
    y = torch.empty((b, 4), dtype=torch.float32, device="cuda")
    ks.ks_mlp_forward(_dev(p), _dev(x), y)
    g = torch.empty(M.NP, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ks.ks_mlp_grad(_dev(p), _dev(x), _dev(t), _dev(mask), g, loss)
    torch.cuda.synchronize()
    y_ref, _ = M.forward(p, x)
    L_ref, g_ref = M.loss_and_grad(p, x, t, mask)
    assert np.allclose(y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-5)
    assert abs(float(loss.item()) - L_ref) <= 1e-5 + 1e-4 * abs(L_ref)
    gg = g.cpu().numpy().astype(np.float64)
    bad = np.abs(gg - g_ref) > 1e-5 + 1e-3 * np.abs(g_ref)
    assert not bad.any(), f"{bad.sum()} gradient entries off, first {np.argwhere(bad)[:3].ravel()}"


@pytest.mark.parametrize("b", [64, 600])
def test_mlp_training_step_is_adam_on_oracle_gradient(b):
    """One ks_mlp_train step equals Adam applied to the oracle's gradient (600 rows: the
    rows pass through shared memory in three chunks)."""
    import torch
    p, x, t, mask = _case(3, b)
    dp, m, v, g = _dev(p.copy()), _dev(np.zeros(M.NP, np.float32)), \
        _dev(np.zeros(M.NP, np.float32)), _dev(np.zeros(M.NP, np.float32))
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ks.ks_mlp_train(dp, m, v, g, _dev(x), _dev(t), _dev(mask), 1, 1e-2, 0, loss)
    torch.cuda.synchronize()
    _, gr = M.loss_and_grad(p, x, t, mask)
    mh = 0.1 * gr / (1 - 0.9)
    vh = 0.001 * gr * gr / (1 - 0.999)
    want = p - 1e-2 * mh / (np.sqrt(vh) + 1e-8)
    assert np.allclose(dp.cpu().numpy(), want, rtol=1e-4, atol=2e-6)


def test_mlp_training_fits_a_smooth_target():
    import torch
    g = np.random.default_rng(5)
    x = g.normal(0, 1, size=(200, 6)).astype(np.float32)
    t = np.stack([np.sin(x[:, 0]) + x[:, 1], x[:, 2] * x[:, 3], np.abs(x[:, 4]), x[:, 5] ** 2],
                 1).astype(np.float32)
    p = _dev(S.init_params(0))
    z = lambda: _dev(np.zeros(M.NP, np.float32))  # noqa: E731
    loss = torch.empty(3000, dtype=torch.float32, device="cuda")
    ks.ks_mlp_train(p, z(), z(), z(), _dev(x), _dev(t), _dev(np.ones_like(t)), 3000, 3e-3, 0, loss)
    torch.cuda.synchronize()
    ls = loss.cpu().numpy()
    assert ls[-1] < 0.05 * ls[0] and ls[-1] < 0.05


SWEEP = os.path.join(S.DATA, "sweep_gb300.json")


@pytest.mark.skipif(not os.path.exists(SWEEP), reason="no committed GB300 sweep")
def test_selector_gain_on_held_out_points():
    data = S.load_json(SWEEP)
    tr, te = S.split(len(data["points"]))
    assert len(te) == 40 and len(tr) == len(data["points"]) - 40
    sel, losses = S.train(data, tr)
    assert losses[-1] < losses[0]
    ev = S.evaluate(data, sel, te, tr)
    fixed = [k for k in ev if k.startswith("fixed_")][0]
    mlp = ev["mlp"]["mean_regret"]
    # what the network gains over the methods without it
    print(ev)
    assert mlp < ev[fixed]["mean_regret"], ev
    assert mlp < ev["footprint_rule"]["mean_regret"], ev
    assert ev["mlp"]["total_ms"] < ev[fixed]["total_ms"], ev
    assert mlp <= 0.05, ev
    # the one-line rule (radix 4 up to N = 2^15, DPOB throughout) is within a few percent
    # of exhaustive on top-level points; the network must stay close to it there
    assert mlp <= ev["threshold_rule"]["mean_regret"] + 0.01, ev
    # the held-out points' lower levels (level views): the network picks per level, where
    # the rule misses (few digits, small L) and the network must beat it
    if "levels" in ev:
        lv = ev["levels"]
        assert lv["mlp"]["mean_regret"] < lv[fixed]["mean_regret"], lv
        assert lv["mlp"]["total_ms"] < lv[fixed]["total_ms"], lv
        assert lv["mlp"]["mean_regret"] < lv["threshold_rule"]["mean_regret"], lv
        assert lv["mlp"]["mean_regret"] <= 0.05, lv


def test_binding_rejects_strided_tensors():
    """A transposed view would be read in the wrong order by the kernels: refused."""
    import torch
    x = torch.zeros((4, 6), dtype=torch.float32, device="cuda").t()
    y = torch.empty((6, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        ks.ks_mlp_forward(_dev(S.init_params(0)), x, y)


@pytest.mark.skipif(not os.path.exists(SWEEP), reason="no committed GB300 sweep")
def test_library_selector_matches_python_and_plans_a_batch():
    """The network installed in the library (ks_selector_load) picks, through ks_select,
    the plan the Python selector picks for the same workload (same kernel, features and
    decoding), for top-level contexts and level views; a KS_BATCH_SELECT batch runs the
    picked plans and stays bit-exact against the oracle."""
    import torch
    from oracle import oracle as O
    data = S.load_json(SWEEP)
    tr, te = S.split(len(data["points"]))
    sel, _ = S.train(data, tr, steps=1500)
    sel.install()
    for i in te[:10]:
        prm = W.make_params(*data["points"][i])
        ctx = ks.Context(prm)
        try:
            want = S.CANDS[sel.choose([prm])[0]]
            assert ks.ks_select(ctx.h) == (want[1], want[2]), (prm.name(), want[0])
            assert ks.ks_context_info(ctx.h)["selected_variant"] == want[1]
            lv = prm.L // 2
            view = ctx.at_level(lv)
            try:
                want = S.CANDS[sel.choose([S.level_shape(prm, lv)])[0]]
                assert ks.ks_select(view.h) == (want[1], want[2]), (prm.name(), lv, want[0])
            finally:
                view.close()
        finally:
            ctx.close()
    # a batch of jobs naming KS_AUTO, planned by the installed network; (3, 2^16, 11)
    # runs its pick with the tensor-core conversions added (N >= 2^16, three digits)
    cfgs = [(2, 13, 7), (3, 14, 11), (2, 13, 7), (5, 12, 9), (3, 16, 11)]
    ctxs, arg, want = {}, [], []
    try:
        for k, cfg in enumerate(cfgs):
            prm = W.make_params(*cfg)
            if cfg not in ctxs:
                ctxs[cfg] = ks.Context(prm)
            g = W.rng(300 + k, 13)
            d = W.uniform_limbs(g, prm.q, prm.N)
            evk = W.uniform_limbs(g, prm.mods * (2 * prm.beta), prm.N).reshape(
                prm.beta, 2, prm.QP, prm.N)
            out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device="cuda")
            arg.append((ctxs[cfg].h, _dev(d), _dev(evk), out))
            want.append(O.keyswitch(prm, d, evk))
        for flags in (ks.KS_BATCH_SELECT, ks.KS_BATCH_SELECT | ks.KS_BATCH_GRAPH):
            for _, _, _, out in arg:
                out.fill_(5)
            ks.ks_switch_batch(arg, flags)
            torch.cuda.synchronize()
            for k, (_, _, _, out) in enumerate(arg):
                assert np.array_equal(out.cpu().numpy(), want[k]), (flags, cfgs[k])
        for cfg, c in ctxs.items():
            prm = W.make_params(*cfg)
            info = ks.ks_context_info(c.h)
            v, ch = info["selected_variant"], info["selected_chunks"]
            assert v == S.CANDS[sel.choose([prm])[0]][1]
            # the plan KS_AUTO runs: the pick, plus KS_BCONV_TC where the rule adds it
            tc = info["tc"] and prm.N >= 1 << 16 and prm.L + 1 > prm.alpha
            assert tc == (cfg == (3, 16, 11))
            runs = v | (ks.KS_BCONV_TC if tc else 0)
            assert ks.ks_workspace_size(c.h, ks.KS_AUTO, 0) == ks.ks_workspace_size(c.h, runs, ch)
        with pytest.raises(ks.KSError):
            ks.ks_switch_batch(arg, ks.KS_BATCH_SELECT | ks.KS_BATCH_AUTOTUNE)
    finally:
        for c in ctxs.values():
            c.close()


def test_selector_load_rejects_bad_networks():
    p = S.init_params(0)
    ok = dict(x_mean=[0.0] * 6, x_std=[1.0] * 6, t_mean=[0.0] * 4, t_std=[1.0] * 4,
              plans=[(v, c) for _, v, c in S.CANDS])
    for bad in (dict(x_std=[1.0] * 5 + [0.0]), dict(t_std=[1.0, -1.0, 1.0, 1.0]),
                dict(plans=[(9, 0)] + ok["plans"][1:]),
                dict(plans=[(ks.KS_DPOB | ks.KS_RADIX4 | ks.KS_RADIX16, 0)] + ok["plans"][1:])):
        with pytest.raises(ks.KSError):
            ks.ks_selector_load(p, **{**ok, **bad})
    q = p.copy()
    q[7] = np.nan
    with pytest.raises(ks.KSError):
        ks.ks_selector_load(q, **ok)
