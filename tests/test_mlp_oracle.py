"""Pins of the selector-MLP oracle: its gradient equals central finite differences of
its loss (float64), and its layout matches the library's constant."""
import numpy as np

from oracle import mlp_oracle as M


def _case(seed, b=24):
    g = np.random.default_rng(seed)
    p = g.normal(0, 0.3, size=M.NP)
    x = g.normal(0, 1, size=(b, M.IN))
    t = g.normal(0, 1, size=(b, M.OUT))
    mask = (g.random((b, M.OUT)) < 0.8).astype(np.float64)
    return p, x, t, mask


def test_layout_size():
    assert M.NP == 4868


def test_gradient_matches_finite_differences():
    p, x, t, mask = _case(0)
    L, g = M.loss_and_grad(p, x, t, mask)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(M.NP, 200, replace=False),
                          [0, 383, 384, 447, 448, 4543, 4544, 4607, 4608, 4863, 4864, 4867]])
    h = 1e-6
    for k in idx:
        e = np.zeros(M.NP)
        e[k] = h
        fd = (M.loss_and_grad(p + e, x, t, mask)[0] - M.loss_and_grad(p - e, x, t, mask)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-5 * abs(fd), (k, fd, g[k])


def test_masked_entries_do_not_contribute():
    p, x, t, mask = _case(2)
    mask[:, 1] = 0
    t2 = t.copy()
    t2[:, 1] += 100.0
    assert np.allclose(M.loss_and_grad(p, x, t, mask)[1], M.loss_and_grad(p, x, t2, mask)[1])


def test_selector_target_encoding_round_trips():
    """Output 0 is the first candidate's log-latency, the others are log-ratios to it."""
    from paper_2603_16692_gb300 import selector as S
    g = np.random.default_rng(3)
    L = np.log(g.uniform(0.01, 10.0, size=(7, 4)))
    E = S.encode(L)
    assert np.allclose(E[:, 0], L[:, 0])
    assert np.allclose(E[:, 1:], L[:, 1:] - L[:, :1])
    assert np.allclose(S.decode(E), L)


def test_level_shape_matches_the_level_view():
    """A KeySwitch at level l keeps alpha and has ceil((l+1)/alpha) digits over
    l+1+alpha limbs; at the top level it is the context's own shape."""
    from paper_2603_16692_gb300 import selector as S
    from paper_2603_16692_gb300 import workload as W
    prm = W.make_params(4, 16, 35)
    top = S.level_shape(prm, prm.L)
    assert (top.beta, top.QP, top.N) == (prm.beta, prm.QP, prm.N)
    assert S.features(top, 1 << 27)[3:] == S.features(prm, 1 << 27)[3:]
    low = S.level_shape(prm, 10)
    assert (low.beta, low.QP, low.dnum) == (2, 20, 2)


def test_selector_features_follow_the_working_set_definitions():
    """The six features of a workload (the library computes the same in ks_select):
    log2 N, L+1, dnum (digits for a level view), and log2 of the DPOB ModUp working set
    beta*QP*N*8, the DSOB one QP*N*8 and the key bytes 2*beta*QP*N*8 over the L2 size;
    here at (2, 2^15, 10) (alpha = 6, beta = 2, QP = 17) against a 2^27-byte L2."""
    import math
    from paper_2603_16692_gb300 import selector as S
    from paper_2603_16692_gb300 import workload as W
    prm = W.make_params(2, 15, 10)
    f = S.features(prm, 1 << 27)
    n8 = (1 << 15) * 8
    assert f[:3] == [15, 11, 2]
    assert f[3] == math.log2(2 * 17 * n8 / (1 << 27))
    assert f[4] == math.log2(17 * n8 / (1 << 27))
    assert f[5] == f[3] + 1.0
    # a level view: 5 Q-limbs of a dnum-2 context keep alpha = 6, so one digit
    lv = S.features(S.level_shape(prm, 4), 1 << 27)
    assert lv[:3] == [15, 5, 1]
    assert lv[4] == math.log2((5 + 6) * n8 / (1 << 27))
