"""Learned dataflow selector (the parameter-aware choice the paper proposes in Sec. V).

A 6 -> 64 -> 64 -> 4 FP32 MLP predicts the latency of four candidate plans from
workload features; the selected plan is the argmin. The candidates are the plans
that compete on GB300 in the library's own sweep of ten plans (four dataflows x
radix 8 / radix 4, OutputChunked with 2 and 4 chunks): DPOB, DSOB, DPOB with
radix-4 rounds, and DPOC with 2 chunks. Output 0 is the log-latency of DPOB,
outputs 1-3 the log-ratios of the other candidates to it (each output standardised
over the training rows): the latencies span three orders of magnitude across
workloads while the choice depends on differences of a few percent, which an
absolute-log target leaves almost unweighted. Training and inference run in the
library's CUDA kernels (ks_mlp_train, ks_mlp_forward). Exhaustive timing of all
ten plans stays the fallback and the yardstick of the regret. The selector never touches
the KeySwitch arithmetic.

Features of (dnum, N, L) on a GPU with L2 bytes: log2 N, L+1, dnum, and log2 of
(DPOB footprint / L2), (DSOB footprint / L2), (evk bytes / L2), where the
footprints are the ModUp working sets of Table III (beta*QP*N*8 and QP*N*8 bytes).
"""
from __future__ import annotations

import dataclasses
import json
import math
import os

import numpy as np

from . import ks
from . import workload as W

CANDS = [("DPOB", ks.KS_DPOB, 0), ("DSOB", ks.KS_DSOB, 0),
         ("DPOB-r4", ks.KS_DPOB | ks.KS_RADIX4, 0), ("DPOC-c2", ks.KS_DPOC, 2)]


def encode(log_ms: np.ndarray) -> np.ndarray:
    """Targets from candidate log-latencies: [log t_0, log t_k - log t_0 (k >= 1)]."""
    return np.concatenate([log_ms[:, :1], log_ms[:, 1:] - log_ms[:, :1]], axis=1)


def decode(enc: np.ndarray) -> np.ndarray:
    """Candidate log-latencies from network outputs (inverse of encode)."""
    return np.concatenate([enc[:, :1], enc[:, 1:] + enc[:, :1]], axis=1)


DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


@dataclasses.dataclass(frozen=True)
class LevelShape:
    """The shape of a KeySwitch at level l of a context (a level view): l+1 Q-limbs,
    the context's alpha special primes, beta_l = ceil((l+1)/alpha) digits. It has the
    attributes `features` reads, with the number of digits in the role of dnum, so the
    selector can pick a plan per level (Sec. V: switch the dataflow as L falls)."""
    logn: int
    L: int
    alpha: int

    @property
    def N(self):
        return 1 << self.logn

    @property
    def beta(self):
        return -(-(self.L + 1) // self.alpha)

    @property
    def dnum(self):
        return self.beta

    @property
    def QP(self):
        return self.L + 1 + self.alpha


def level_shape(prm, level: int) -> LevelShape:
    return LevelShape(prm.logn, level, prm.alpha)


def footprints(prm) -> dict:
    """ModUp working-set bytes of each dataflow (Table III: O(dNL), O(NL), O(NL/c), O(dNL/c))."""
    n8 = prm.N * 8
    return {"DPOB": prm.beta * prm.QP * n8, "DSOB": prm.QP * n8,
            "DSOC-c2": -(-prm.QP // 2) * n8, "DPOC-c2": prm.beta * -(-prm.QP // 2) * n8,
            "DPOC-c4": prm.beta * -(-prm.QP // 4) * n8}


def features(prm, l2: int) -> list:
    fp = footprints(prm)
    evk = 2 * prm.beta * prm.QP * prm.N * 8
    return [prm.logn, prm.L + 1, prm.dnum, math.log2(fp["DPOB"] / l2), math.log2(fp["DSOB"] / l2),
            math.log2(evk / l2)]


def footprint_rule(prm, l2: int) -> int:
    """The paper's rule (Sec. IV-B): the best strategy moves to the next smaller footprint
    once L2 is below about twice the footprint. Over the candidate dataflows (radix 8),
    by decreasing footprint: the first with 2 x footprint <= L2, else the smallest."""
    fp = footprints(prm)
    ks_ = [k for k, (n, v, c) in enumerate(CANDS) if not v & ks.KS_RADIX4]
    order = sorted(ks_, key=lambda k: -fp[CANDS[k][0]])
    for k in order:
        if 2 * fp[CANDS[k][0]] <= l2:
            return k
    return order[-1]


def threshold_rule(prm, l2: int = 0) -> int:
    """A one-line rule read off the GB300 sweep: DPOB with radix-4 rounds up to
    N = 2^15, DPOB with radix-8 rounds above (the baseline the network must beat)."""
    return 2 if prm.N <= 1 << 15 else 0


def columns(data: dict) -> list:
    """Indices of the candidate plans among the sweep's measured plans."""
    return [data["cands"].index(n) for n, _, _ in CANDS]


# ---------------------------------------------------------------------------
# Sweep: time every candidate on each point through the library.

ALL_PLANS = [(f"{n}{'-r4' if r4 else ''}", v | (ks.KS_RADIX4 if r4 else 0), c)
             for n, v, c in [("DSOB", ks.KS_DSOB, 0), ("DPOB", ks.KS_DPOB, 0),
                             ("DSOC-c2", ks.KS_DSOC, 2), ("DPOC-c2", ks.KS_DPOC, 2),
                             ("DPOC-c4", ks.KS_DPOC, 4)] for r4 in (0, 1)]


def sweep_levels(L: int) -> list:
    """The lower levels measured beside a top-level point: L/2 and L/5 (rounded down,
    distinct, below L)."""
    return sorted({lv for lv in (L // 2, L // 5) if 0 <= lv < L})


def sweep(points, reps: int = 5, seed: int = 0, log=print, cands=None) -> dict:
    """Median time of each plan on each point (a KeySwitch with random inputs), and on
    the point's lower levels (level views with the point's key: `levels` rows)."""
    import torch
    dev = torch.device("cuda")
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    plans = cands or CANDS

    def rand_limbs(mods, lead, n):
        t = torch.empty((*lead, len(mods), n), dtype=torch.int64, device=dev)
        for i, m in enumerate(mods):
            t[..., i, :] = torch.randint(0, m, (*lead, n), generator=gen, device=dev,
                                         dtype=torch.int64)
        return t.view(torch.uint64)

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def measure(h, d, evk, out):
        row = []
        for name, v, c in plans:
            for _ in range(2):
                ks.ks_switch(h, d, evk, out, v, c, None, stream)
            ts = []
            for _ in range(reps):
                e0.record(stream)
                ks.ks_switch(h, d, evk, out, v, c, None, stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            row.append(float(np.median(ts)))
        return row

    ms, levels, level_ms = [], [], []
    for k, cfg in enumerate(points):
        prm = W.make_params(*cfg)
        ctx = ks.Context(prm)
        evk = rand_limbs(prm.mods, (prm.beta, 2), prm.N)
        d = rand_limbs(prm.q, (), prm.N)
        out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device=dev)
        row = measure(ctx.h, d, evk, out)
        ms.append(row)
        for lv in sweep_levels(prm.L):
            view = ctx.at_level(lv)
            dl = rand_limbs(prm.q[:lv + 1], (), prm.N)
            ol = torch.empty((2, lv + 1, prm.N), dtype=torch.uint64, device=dev)
            levels.append([k, lv])
            level_ms.append(measure(view.h, dl, evk, ol))
            view.close()
        ctx.close()
        del d, evk, out
        if log and (k % 20 == 0 or k == len(points) - 1):
            log(f"sweep {k + 1}/{len(points)} {cfg}: " +
                " ".join(f"{n}={t:.3f}ms" for (n, _, _), t in zip(plans, row)))
    torch.cuda.empty_cache()
    return {"device": torch.cuda.get_device_name(dev), "l2": int(l2), "reps": reps,
            "cands": [n for n, _, _ in plans], "points": [list(p) for p in points],
            "ms": ms, "levels": levels, "level_ms": level_ms}


def shapes_and_times(data: dict, idx):
    """(shapes, times[rows][plans]) of the top-level points idx and of their level rows
    (a sweep without level rows gives the points alone)."""
    pts = [W.make_params(*data["points"][i]) for i in idx]
    ms = [data["ms"][i] for i in idx]
    keep = set(idx)
    for (k, lv), row in zip(data.get("levels", []), data.get("level_ms", [])):
        if k in keep:
            pts.append(level_shape(W.make_params(*data["points"][k]), lv))
            ms.append(row)
    return pts, np.array(ms, dtype=np.float64)


def split(n: int, n_test: int = 40, seed: int = 0):
    """Seeded split of the sweep into train and held-out indices."""
    g = W.rng(seed, 5)
    perm = g.permutation(n)
    return sorted(perm[n_test:].tolist()), sorted(perm[:n_test].tolist())


# ---------------------------------------------------------------------------
# Model

class Selector:
    def __init__(self, params, x_mean, x_std, t_mean, t_std, l2):
        self.params = np.asarray(params, dtype=np.float32)
        self.x_mean = np.asarray(x_mean, dtype=np.float64)
        self.x_std = np.asarray(x_std, dtype=np.float64)
        self.t_mean = np.asarray(t_mean, dtype=np.float64)  # per output
        self.t_std = np.asarray(t_std, dtype=np.float64)
        self.l2 = int(l2)

    def norm_x(self, feats) -> np.ndarray:
        return ((np.asarray(feats, dtype=np.float64) - self.x_mean) / self.x_std).astype(np.float32)

    def predict_ms(self, prms) -> np.ndarray:
        """Predicted latency (ms) of each candidate, on the GPU (ks_mlp_forward)."""
        import torch
        x = torch.from_numpy(np.ascontiguousarray(
            self.norm_x([features(p, self.l2) for p in prms]))).cuda()
        p = torch.from_numpy(self.params).cuda()
        y = torch.empty((len(prms), 4), dtype=torch.float32, device="cuda")
        for s in range(0, len(prms), ks.KS_MLP_MAX_BATCH):
            xs = x[s:s + ks.KS_MLP_MAX_BATCH].contiguous()
            ys = torch.empty((xs.shape[0], 4), dtype=torch.float32, device="cuda")
            ks.ks_mlp_forward(p, xs, ys)
            y[s:s + xs.shape[0]] = ys
        torch.cuda.synchronize()
        return np.exp(decode(y.cpu().numpy().astype(np.float64) * self.t_std + self.t_mean))

    def choose(self, prms) -> list:
        return [int(k) for k in np.argmin(self.predict_ms(prms), axis=1)]

    def install(self):
        """Installs this network in the library (ks_selector_load): ks_select and
        ks_switch_batch with KS_BATCH_SELECT then pick plans without Python."""
        ks.ks_selector_load(self.params, self.x_mean, self.x_std, self.t_mean, self.t_std,
                            [(v, c) for _, v, c in CANDS], self.l2)

    def to_json(self) -> dict:
        return {"params": self.params.tolist(), "x_mean": self.x_mean.tolist(),
                "x_std": self.x_std.tolist(), "t_mean": self.t_mean.tolist(),
                "t_std": self.t_std.tolist(), "l2": self.l2, "cands": [n for n, _, _ in CANDS]}

    @staticmethod
    def from_json(d) -> "Selector":
        return Selector(d["params"], d["x_mean"], d["x_std"], d["t_mean"], d["t_std"], d["l2"])


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation of the 6-64-64-4 layout (seeded)."""
    g = np.random.default_rng(seed)
    parts = [g.normal(0, math.sqrt(2 / 6), 6 * 64), np.zeros(64),
             g.normal(0, math.sqrt(2 / 64), 64 * 64), np.zeros(64),
             g.normal(0, math.sqrt(1 / 64), 64 * 4), np.zeros(4)]
    return np.concatenate(parts).astype(np.float32)


def train(data: dict, idx, steps: int = 4000, lr: float = 3e-3, seed: int = 0):
    """Fit the MLP on the sweep rows `idx` with the library's CUDA training kernel.
    Returns (Selector, per-step losses)."""
    import torch
    shapes, times = shapes_and_times(data, idx)
    l2 = data["l2"]
    X = np.array([features(p, l2) for p in shapes], dtype=np.float64)
    cols = columns(data)
    T = encode(np.log(times[:, cols]))
    x_mean, x_std = X.mean(0), X.std(0) + 1e-9
    t_mean, t_std = T.mean(0), T.std(0) + 1e-9
    sel = Selector(init_params(seed), x_mean, x_std, t_mean, t_std, l2)
    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(sel.norm_x(X))).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(((T - t_mean) / t_std).astype(np.float32))).to(dev)
    mask = torch.ones_like(t)
    p = torch.from_numpy(sel.params.copy()).to(dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.zeros_like(p)
    loss = torch.zeros(steps, dtype=torch.float32, device=dev)
    ks.ks_mlp_train(p, m, v, g, x, t, mask, steps, lr, 0, loss)
    torch.cuda.synchronize()
    sel.params = p.cpu().numpy()
    return sel, loss.cpu().numpy()


def fixed_choice(data: dict, train_idx) -> int:
    """The best single fixed candidate on the training rows (least total time)."""
    _, tr_times = shapes_and_times(data, train_idx)
    return int(np.argmin(tr_times[:, columns(data)].sum(0)))


def score(sel: Selector, shapes, times, cols, fixed: int, l2: int) -> dict:
    """Regret t(chosen)/t(best) - 1 per row, the best being the exhaustive minimum over
    every measured plan (times[rows][plans]; cols = the candidates' columns), for the
    MLP, the fixed candidate, the paper's footprint rule and the one-line threshold
    rule."""
    times = np.asarray(times, dtype=np.float64)
    best = times.min(1)
    ms = times[:, cols]
    res = {}
    for name, ch in (("mlp", sel.choose(shapes)),
                     ("fixed_" + CANDS[fixed][0], [fixed] * len(shapes)),
                     ("footprint_rule", [footprint_rule(p, l2) for p in shapes]),
                     ("threshold_rule", [threshold_rule(p) for p in shapes])):
        r = np.array([ms[i, c] / best[i] - 1 for i, c in enumerate(ch)])
        res[name] = {"mean_regret": float(r.mean()), "max_regret": float(r.max()),
                     "total_ms": float(sum(ms[i, c] for i, c in enumerate(ch)))}
    res["exhaustive_total_ms"] = float(best.sum())
    return res


def evaluate(data: dict, sel: Selector, test_idx, train_idx) -> dict:
    """Regret on the held-out points test_idx of the sweep `data` (and, under "levels",
    on their lower levels if the sweep has them); see score()."""
    fixed = fixed_choice(data, train_idx)
    cols = columns(data)
    top = [W.make_params(*data["points"][i]) for i in test_idx]
    out = score(sel, top, [data["ms"][i] for i in test_idx], cols, fixed, data["l2"])
    shapes, times = shapes_and_times(data, test_idx)
    if len(shapes) > len(top):
        out["levels"] = dict(score(sel, shapes[len(top):], times[len(top):], cols, fixed,
                                   data["l2"]), rows=len(shapes) - len(top))
    return out


def evaluate_live(live: dict, sel: Selector, fixed: int) -> dict:
    """Regret judged on a sweep `live` re-timed now (every plan of ALL_PLANS on the
    held-out points and their lower levels), with the network and the fixed candidate
    chosen from the training sweep."""
    idx = list(range(len(live["points"])))
    cols = columns(live)
    top = [W.make_params(*p) for p in live["points"]]
    out = score(sel, top, live["ms"], cols, fixed, live["l2"])
    shapes, times = shapes_and_times(live, idx)
    if len(shapes) > len(top):
        out["levels"] = dict(score(sel, shapes[len(top):], times[len(top):], cols, fixed,
                                   live["l2"]), rows=len(shapes) - len(top))
    return out


def load_json(path):
    with open(path) as f:
        return json.load(f)


def save_json(path, obj):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(obj, f)


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="selector sweep / training")
    ap.add_argument("cmd", choices=["sweep", "train"])
    ap.add_argument("--points", type=int, default=200)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--data", default=os.path.join(DATA, "sweep_gb300.json"))
    ap.add_argument("--model", default=os.path.join(DATA, "selector_gb300.json"))
    a = ap.parse_args()
    if a.cmd == "sweep":
        save_json(a.data, sweep(W.selector_points(0, a.points), a.reps, cands=ALL_PLANS))
    else:
        data = load_json(a.data)
        tr, te = split(len(data["points"]))
        sel, losses = train(data, tr)
        save_json(a.model, sel.to_json())
        print(json.dumps({"final_loss": float(losses[-1]), **evaluate(data, sel, te, tr)}))
