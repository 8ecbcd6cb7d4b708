#!/usr/bin/env python3
"""KeySwitch throughput benchmark: one JSON line on rank 0.

A step is one hybrid KeySwitch (iNTT, ModUp BConv + NTT, key multiply, iNTT,
ModDown BConv + NTT, P^-1 scaling) of the workload's input polynomial, launched
through the C-ABI (ks_switch) on device-resident buffers. Each step uses the
next (d, evk, out) set from a ring of distinct buffers larger than twice the L2
cache, so every step reads its inputs from HBM. Independent steps run on up to
three streams in flight, each with its own workspace (the count measured fastest on
a short probe); the one-stream rate is reported beside it.

Default workload: plain KeySwitch (dnum, N, L) = (4, 2^16, 35), the configuration
the HBM-roofline target is stated on; --workload c1 / c2 selects (2, 2^13, 7) or
(2, 2^15, 10). With --gpus N > 1
(torchrun, one process per GPU) every rank runs an independent replica: the
KeySwitches of different ranks share nothing ("replicas only", weak scaling).

--impl reference times the plain CPU oracle instead (the baseline the CUDA path
is checked against), on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2603_16692_gb300 import workload as W  # noqa: E402

METRIC = "KeySwitch/s per (dnum,N,L) on 1 GB300, % HBM roofline, selector regret"
MAX_STREAMS = 3
UNIT = "KeySwitch/s"
WORKLOADS = {"c1": W.C1, "c2": W.C2, "c3": W.C3}

# Per-kernel DRAM bytes (read + write) per launch and pipe use, from the cold-cache ncu
# launch list and the per-kernel --set full captures of one KeySwitch of the workload
# (profile_case; summaries and commands in profiles/keyswitch_4_2e16_35_launches.md,
# keyswitch_4_2e16_35_kernels_ncu.md and bconv_tc_4_2e16_35_ncu.md), one table per
# captured plan, keyed by the kernel names of the library's profiler, so a change of the
# dominant kernel still finds its row. In the split plan the key multiply's two launches
# (P-limb and Q-limb targets) are averaged, as the profiler averages them. The integer
# plan DPOB[km4,dnr4]-split and the tensor-core plan DPOB[km4]-tc (KS_BCONV_TC); pipe
# use where a --set full capture exists.
NCU_PLANS = {
    ("c3", "DPOB[km4,dnr4]-split"): {k: {"traffic": t, **pipes} for k, t, pipes in (
        ("intt_row(d)", 57100000, {"issue_pct": 47.3, "fmaheavy_pct": 45.0, "alu_pct": 37.3}),
        ("intt_col(d)", 19100000, {"issue_pct": 45.8, "fmaheavy_pct": 47.0, "alu_pct": 35.0}),
        ("modup_col", 38400000, {"issue_pct": 59.8, "fmaheavy_pct": 69.0, "alu_pct": 48.3}),
        ("modup_row_keymult", 176050000,
         {"issue_pct": 54.1, "fmaheavy_pct": 55.0, "alu_pct": 37.2}),
        ("intt_row(accP)", 18900000, {"issue_pct": 45.2, "fmaheavy_pct": 38.0, "alu_pct": 38.6}),
        ("intt_col(accP)", 9500000, {"issue_pct": 45.0, "fmaheavy_pct": 41.0, "alu_pct": 37.1}),
        ("moddown_col", 9600000, {"issue_pct": 58.2, "fmaheavy_pct": 66.0, "alu_pct": 46.0}),
        ("moddown_row", 123700000, {"issue_pct": 51.7, "fmaheavy_pct": 52.0, "alu_pct": 44.7}))},
    ("c3", "DPOB[km4]-tc"): {k: {"traffic": t, **pipes} for k, t, pipes in (
        ("intt_row(d)", 57050000, {}),
        ("intt_col(d)", 19080000, {}),
        ("modup_col", 108350000,
         {"issue_pct": 41.3, "tensor_pct": 8.9, "alu_pct": 29.1, "fma_pct": 27.9}),
        ("modup_row_keymult", 361500000, {}),
        ("intt_row(accP)", 18880000, {}),
        ("intt_col(accP)", 9520000, {}),
        ("moddown_col", 19190000,
         {"issue_pct": 41.1, "tensor_pct": 9.1, "alu_pct": 28.5, "fma_pct": 27.5}),
        ("moddown_row", 126320000, {}))},
}
# the column-pass kernels whose code depends on the tensor-core flags: a row for another
# plan with the same flags stands for them (the other kernels' traffic depends on the
# plan's split and schedule)
TC_KERNELS = {"intt_col(d)": "up", "modup_col": "up", "intt_col(accP)": "down",
              "moddown_col": "down"}


def ncu_row(workload, plan, name, tc_up, tc_down):
    """The ncu row of kernel `name` of plan `plan` (its variant name): the captured plan
    itself, else, for the tensor-core-dependent column kernels, the captured plan with
    the same conversion on the same kind of pipe; None when there is no such capture.
    tc_up / tc_down: the plan's ModUp / ModDown conversions run on the tensor cores."""
    rows = NCU_PLANS.get((workload, plan))
    if rows and name in rows:
        return {"plan": plan, **rows[name]}
    side = TC_KERNELS.get(name)
    if side:
        tc = tc_up if side == "up" else tc_down
        ref = "DPOB[km4]-tc" if tc else "DPOB[km4,dnr4]-split"
        row = NCU_PLANS.get((workload, ref), {}).get(name)
        if row:
            return {"plan": ref, **row}
    return None


def tc_sides(ks, variant):
    """(ModUp, ModDown) conversions of a plan on the tensor cores."""
    return (bool(variant & ks.KS_BCONV_TC),
            bool(variant & (ks.KS_BCONV_TC | ks.KS_BCONV_TC_DOWN)))


def measured_alu(ks, stream):
    """The library's measured arithmetic ceiling on this GPU: its own butterfly and
    128-bit multiply-accumulate kernels at full occupancy with no memory traffic."""
    bf = max(ks.ks_calibrate(ks.KS_CAL_BUTTERFLY, 16384, stream) for _ in range(3))
    mac = max(ks.ks_calibrate(ks.KS_CAL_MAC, 4096, stream) for _ in range(3))
    return bf, mac


def tensor_roofline(dom, per_launch_ms, peaks):
    """The tensor-core part of a kernel (the basis conversions of KS_BCONV_TC plans), or
    None: its bf16 FLOPs against the measured sustained cuBLAS bf16 rate (the kernel runs
    inside a long step)."""
    if not dom.get("tensor_flops"):
        return None
    fl = dom["tensor_flops"] / dom["launches"]
    pk = float(peaks.get("bf16_tflops_sustained", 1700.0)) * 1e12
    return {"flops_per_launch": fl, "achieved": fl / (per_launch_ms / 1e3) / 1e12,
            "peak": pk / 1e12, "unit": "TFLOP/s", "frac": fl / pk * 1e3 / per_launch_ms,
            "t_ceil_ms": fl / pk * 1e3,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained" if
            "bf16_tflops_sustained" in peaks else "fallback 1.7 PFLOP/s sustained"}


def alu_roofline(dom, per_launch_ms, bf, mac):
    """A kernel against the measured ceiling of its own arithmetic. Its MAC terms are
    converted to butterfly-equivalents at the measured rate ratio, so achieved / peak
    = t_ceil / t with t_ceil = MACs / mac_rate + Shoup products / butterfly_rate."""
    n = dom["launches"]
    macs, shoup = dom["macs"] / n, (dom["ops"] - dom["macs"]) / n
    t_ceil_ms = (macs / mac + shoup / bf) * 1e3
    eq_ops = shoup + macs * bf / mac
    return {"achieved": eq_ops / (per_launch_ms / 1e3) / 1e9, "peak": bf / 1e9,
            "frac": t_ceil_ms / per_launch_ms, "t_ceil_ms": t_ceil_ms,
            "macs_per_launch": macs, "shoup_per_launch": shoup}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c3")
    ap.add_argument("--variant", default="tuned",
                    help="tuned (ks_tune picks), or DSOB/DPOB/DSOC/DPOC")
    ap.add_argument("--chunks", type=int, default=0)
    ap.add_argument("--unfused", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bound on the oracle sample (CPU baseline)")
    ap.add_argument("--radix4", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-job uneven batch measurement")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--no-eval", action="store_true",
                    help="skip the HMUL / HROT / level-aware measurements")
    return ap.parse_args()


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def max_over_ranks(x: float, dist, device) -> float:
    """The maximum of x over all ranks of the process group (x with one process)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time
    (ranks are independent replicas, so each processed units_per_rank)."""
    return world * units_per_rank / (ms / 1e3)


def workload_config(prm):
    """The workload, identical on both arms (the plan and the ring's sizes are reported
    beside it, under "plan"); `l2` states how the GPU arm keeps L2 from serving repeated
    inputs."""
    return {"workload": f"plain KeySwitch (dnum,N,L)={prm.name()}", "dnum": prm.dnum,
            "N": prm.N, "L": prm.L, "alpha": prm.alpha, "beta": prm.beta, "QP": prm.QP,
            "qbits": 50, "pbits": 60,
            "l2": "inputs larger than L2: each GPU step switches the next (d, evk, out) set "
                  "of a ring of distinct sets over 2 x L2"}


# ---------------------------------------------------------------------------
# CPU oracle (the reported baseline and the reference arm)

def oracle_sample(prm, seconds: float, max_reps: int, nthreads: int | None = None):
    """Time oracle KeySwitches on `nthreads` host threads (default: all cores) for about
    `seconds` (at least one)."""
    from oracle import oracle as O
    s_from, s_to, a, e = W.gen_keys(prm, 0)
    d = W.gen_input(prm, 0)
    evk = O.keygen(prm, s_from, s_to, a, e)
    O.keyswitch(prm, d, evk, nthreads=nthreads)  # warm (tables, threads)
    reps, t0 = 0, time.perf_counter()
    while reps < max_reps:
        O.keyswitch(prm, d, evk, nthreads=nthreads)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return reps, el, nthreads or O.default_threads()


def run_reference(args, prm, rank: int, world: int):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    one = oracle_sample(prm, 0.0, 1)
    t_one = one[1]
    budget = 90.0
    steps = max(1, min(args.steps, int(budget / max(t_one, 1e-6))))
    # all requested warm-up steps, unless they alone would exceed ~30 s (then >= 3)
    warm = min(args.warmup, max(3, int(30.0 / max(t_one, 1e-6))))
    for _ in range(warm):
        oracle_sample(prm, 0.0, 1)
    reps, el, cores = oracle_sample(prm, 1e9, steps)
    value = reps / el
    sample = f"{reps} of {args.steps} requested steps timed (each one full KeySwitch of the" \
             f" workload, all host threads); capped at ~{budget:.0f} s of CPU work"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": reps, "warmup": warm, "ms_per_step": el / reps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": workload_config(prm),
            "plan": {"variant": "oracle (schoolbook, host cores)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Clock sampling during the timed region

class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100", "-i",
                                       gpu_id], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.windows = []

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [ln.strip().split(", ") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        keep, allrows = [], []
        for r in rows:
            if len(r) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(r[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                sm, smax = float(r[2]), float(r[3])
            except ValueError:
                continue
            allrows.append((ts, sm, smax, r))
            if any(t0 - 1.0 <= ts <= t1 + 1.0 for t0, t1 in self.windows):
                keep.append((ts, sm, smax, r))
        use = keep or allrows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, _, r in use for n, v in zip(names, r[6:10])
                          if v.strip().lower() == "active"})
        return {"sm_mhz": statistics.median(s for _, s, _, _ in use),
                "sm_max_mhz": max(m for _, _, m, _ in use), "reasons": reasons,
                "samples": len(use), "power_w_max": max(float(r[4]) for *_, r in use
                                                        if r[4].replace(".", "").isdigit())
                if any(r[4].replace(".", "").isdigit() for *_, r in use) else None}


# ---------------------------------------------------------------------------
# The uneven batch: 64 KeySwitches, (dnum, N, L) drawn per job from N in 2^13..2^17,
# L in [4, 60], dnum in [2, 10] (seed 0), run as one ks_switch_batch (CUDA graph,
# tuned plans) against the plain form (one ks_switch per job, one fixed dataflow,
# sequential on one stream).

def batch_measure(args, ks, torch, dev, stream, hbm):
    jobs = W.batch_jobs(0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)

    def rand_limbs(mods, lead, n):
        t = torch.empty((*lead, len(mods), n), dtype=torch.int64, device=dev)
        for i, m in enumerate(mods):
            t[..., i, :] = torch.randint(0, m, (*lead, n), generator=gen, device=dev,
                                         dtype=torch.int64)
        return t.view(torch.uint64)

    ctxs, arg, algo = {}, [], 0
    for cfg in jobs:
        prm = W.make_params(*cfg)
        if cfg not in ctxs:
            ctxs[cfg] = ks.Context(prm)
        d = rand_limbs(prm.q, (), prm.N)
        evk = rand_limbs(prm.mods, (prm.beta, 2), prm.N)
        out = torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64, device=dev)
        arg.append((ctxs[cfg].h, d, evk, out))
        algo += prm.algo_bytes()
    torch.cuda.synchronize(dev)

    def timed(fn, reps):
        fn()
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps  # ms per batch

    plain = {}
    for name, v, c in (("DSOB", ks.KS_DSOB, 0), ("DPOB", ks.KS_DPOB, 0),
                       ("DPOC-c4", ks.KS_DPOC, 4), ("DSOC-c2", ks.KS_DSOC, 2)):
        def run_plain(v=v, c=c):
            for h, d, evk, out in arg:
                ks.ks_switch(h, d, evk, out, v, c, None, stream)
        plain[name] = len(jobs) / (timed(run_plain, max(2, args.batch_steps // 4)) / 1e3)
    # learned selector: per-job plans from the MLP (trained on the library's GB300 sweep
    # with the CUDA training kernel), whole batch as one CUDA graph
    from paper_2603_16692_gb300 import selector as S
    sel_info = None
    try:
        data = S.load_json(os.path.join(S.DATA, "sweep_gb300.json"))
        tr, te = S.split(len(data["points"]))
        sel, losses = S.train(data, tr)
        sel_info = S.evaluate(data, sel, te, tr)
        sel_info["train_final_loss"] = float(losses[-1])
        # the regret judged on timings taken now, on this GPU: every plan re-timed on the
        # 40 held-out points and their lower levels
        live = S.sweep([data["points"][i] for i in te], reps=3, cands=S.ALL_PLANS, log=None)
        sel_info["live"] = S.evaluate_live(live, sel, S.fixed_choice(data, tr))
        sel_info["live"]["how"] = f"{len(te)} held-out points + {len(live['levels'])} lower-" \
                                  f"level rows x {len(S.ALL_PLANS)} plans re-timed in this run " \
                                  "(median of 3); network trained on the committed sweep"
        sel_info["sweep"] = f"{len(data['points'])} points (+ {len(data.get('levels', []))} " \
                            f"lower-level rows) x {len(data['cands'])} plans, {len(tr)} train / " \
                            f"{len(te)} held-out points"
        # the network installed in the library plans the batch itself (KS_BATCH_SELECT:
        # one ks_mlp_forward launch per context, then the graph of the picked plans)
        sel.install()
        arg_auto = [(h, d, evk, out, ks.KS_AUTO, 0) for h, d, evk, out in arg]
        sflags = ks.KS_BATCH_GRAPH | ks.KS_BATCH_SELECT
        ms_sel = timed(lambda: ks.ks_switch_batch(arg_auto, sflags, stream), args.batch_steps)
        sel_info["batch_value"] = len(jobs) / (ms_sel / 1e3)
        names = {(v, c): n for n, v, c in S.CANDS}
        lib_picks = [names.get((ks.ks_context_info(h)["selected_variant"],
                                ks.ks_context_info(h)["selected_chunks"]), "?")
                     for h, _, _, _ in arg]
        py_picks = [S.CANDS[k][0] for k in sel.choose([W.make_params(*cfg) for cfg in jobs])]
        sel_info["batch_picks"] = {n: lib_picks.count(n) for n in sorted(set(lib_picks))}
        sel_info["library_picks_match_python"] = lib_picks == py_picks
    except (OSError, ValueError, KeyError) as ex:
        sel_info = {"error": str(ex)}
    flags = ks.KS_BATCH_GRAPH | ks.KS_BATCH_AUTOTUNE
    ms = timed(lambda: ks.ks_switch_batch(arg, flags, stream), args.batch_steps)
    value = len(jobs) / (ms / 1e3)
    # the persistent form (DPOB fused plans): one persistent kernel per stage, replayed
    # from a graph
    pflags = ks.KS_BATCH_PERSISTENT | ks.KS_BATCH_GRAPH
    ms_p = timed(lambda: ks.ks_switch_batch(arg, pflags, stream), args.batch_steps)
    p_status = ks.ks_batch_status(stream)
    best_name = max(plain, key=plain.get)
    tuned = {}
    for c in ctxs.values():
        inf = ks.ks_context_info(c.h)
        name = ks.variant_name(inf["tuned_variant"], inf["tuned_chunks"])
        tuned[name] = tuned.get(name, 0) + 1
    out = {"workload": "64 KeySwitches, (dnum,N,L) per job from N 2^13..2^17, L 4..60, "
                       "dnum 2..10 (seed 0)",
           "value": value, "unit": "KeySwitch/s", "ms_per_batch": ms,
           "form": "one ks_switch_batch call (CUDA graph replay, per-context tuned plans, "
                   "same-shape jobs share launches, contexts on concurrent streams)",
           "plain_ks_per_s": plain, "plain_best_fixed": best_name,
           "speedup_vs_best_fixed": value / plain[best_name],
           "speedup_vs_dsob": value / plain["DSOB"],
           "algo_bytes_per_batch": algo, "hbm_frac": algo / (ms / 1e3) / 1e9 / hbm,
           "tuned_plans": tuned, "selector": sel_info,
           "persistent": {"value": len(jobs) / (ms_p / 1e3), "ms_per_batch": ms_p,
                          "status": ks.strerror(p_status),
                          "speedup_vs_best_fixed": len(jobs) / (ms_p / 1e3) / plain[best_name],
                          "form": "persistent kernels, one per stage over all 64 jobs' "
                                  "tiles (key multiply and ModDown rows in two, by row-tile "
                                  "size), chained by programmatic dependent launch (graph "
                                  "replay)"}}
    if sel_info and "batch_value" in sel_info:
        out["selector_speedup_vs_best_fixed"] = sel_info["batch_value"] / plain[best_name]
    for c in ctxs.values():
        c.close()
    return out


# ---------------------------------------------------------------------------
# The other plain workloads, (2, 2^13, 7) and (2, 2^15, 10): the tuned plan over a ring of
# buffer sets larger than twice L2, device-resident, like the headline.

def other_workloads(names, ks, torch, dev, stream, l2, steps):
    gen = torch.Generator(device=dev)
    gen.manual_seed(99)

    def rand_limbs(mods, lead, n):
        t = torch.empty((*lead, len(mods), n), dtype=torch.int64, device=dev)
        for i, m in enumerate(mods):
            t[..., i, :] = torch.randint(0, m, (*lead, n), generator=gen, device=dev,
                                         dtype=torch.int64)
        return t.view(torch.uint64)

    out = {}
    for name in names:
        prm = W.make_params(*WORKLOADS[name])
        ctx = ks.Context(prm)
        try:
            evk = rand_limbs(prm.mods, (prm.beta, 2), prm.N)
            d = rand_limbs(prm.q, (), prm.N)
            set_bytes = (evk.numel() + 3 * d.numel()) * 8
            ring = max(2, -(-2 * l2 // set_bytes) + 1)
            sets = [(d.clone(), evk.clone(), torch.empty((2, prm.L + 1, prm.N),
                                                         dtype=torch.uint64, device=dev))
                    for _ in range(ring)]
            v, c = ks.ks_tune(ctx.h, sets[0][0], sets[0][1], sets[0][2], 1, stream)
            nws = ks.ks_workspace_size(ctx.h, v, c) // 8 + 1
            strs = [stream] + [torch.cuda.Stream(device=dev) for _ in range(MAX_STREAMS - 1)]
            calls = [[ks.prepare_switch(ctx.h, dd, ee, oo, v, c,
                                        torch.empty(nws, dtype=torch.uint64, device=dev), strs[q])
                      for dd, ee, oo in sets] for q in range(MAX_STREAMS)]
            by_streams = {}
            for ns in range(1, min(MAX_STREAMS, ring) + 1):
                def go(n, ns=ns):
                    for q in range(1, ns):
                        strs[q].wait_stream(stream)
                    for k in range(n):
                        calls[k % ns][k % ring]()
                    for q in range(1, ns):
                        stream.wait_stream(strs[q])
                go(20)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                go(steps)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                by_streams[ns] = e0.elapsed_time(e1) / steps
            ns = min(by_streams, key=by_streams.get)
            ms = by_streams[ns]
            out[name] = {"workload": f"plain KeySwitch (dnum,N,L)={prm.name()}",
                         "plan": ks.variant_name(v, c), "value": 1e3 / ms, "unit": UNIT,
                         "ms_per_step": ms, "steps": steps, "streams_in_flight": ns,
                         "one_stream_value": 1e3 / by_streams[1],
                         "ms_per_step_by_streams": by_streams,
                         "l2": f"ring of {ring} sets > 2 x L2"}
        finally:
            ctx.close()
    return out


# ---------------------------------------------------------------------------
# HMUL and HROT throughput (Sec. II-A: tensor product / Galois automorphism plus a
# KeySwitch), and level-aware switching (Sec. V: re-select the dataflow as the
# level falls): one KeySwitch per level from L down to 0 at (4, 2^16, 35), with one
# fixed plan for every level against the plan ks_tune picks at each level.

def eval_measure(args, ks, torch, dev, stream, l2):
    gen = torch.Generator(device=dev)
    gen.manual_seed(4321)

    def rand_limbs(mods, lead, n):
        t = torch.empty((*lead, len(mods), n), dtype=torch.int64, device=dev)
        for i, m in enumerate(mods):
            t[..., i, :] = torch.randint(0, m, (*lead, n), generator=gen, device=dev,
                                         dtype=torch.int64)
        return t.view(torch.uint64)

    flush = torch.empty(2 * l2 // 8 + 1, dtype=torch.int64, device=dev)

    def per_call_ms(fn, reps):
        """Mean device time of fn() with L2 flushed before every call (flush untimed)."""
        for k in range(2):
            fn(k)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for k, (a, b) in enumerate(evs):
            flush.zero_()
            a.record(stream)
            fn(k)
            b.record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in evs) / reps

    out = {"l2_flushed_between_calls": True}
    reps = 30
    for name, cfg in (("c2", W.C2), ("c3", W.C3)):
        prm = W.make_params(*cfg)
        ctx = ks.Context(prm)
        try:
            keys = [rand_limbs(prm.mods, (prm.beta, 2), prm.N) for _ in range(2)]
            cts = [rand_limbs(prm.q, (2,), prm.N) for _ in range(3)]
            res = torch.empty_like(cts[0])
            k_rot = ks.galois_elt(1, prm.N)
            v, c = ks.ks_tune(ctx.h, cts[0][1].contiguous(), keys[0], res, 1, stream)
            t_ks = per_call_ms(lambda k: ks.ks_switch(ctx.h, cts[k % 3][1], keys[k % 2], res, v,
                                                      c, None, stream), reps)
            t_mul = per_call_ms(lambda k: ks.ks_hmul(ctx.h, cts[k % 3], cts[(k + 1) % 3],
                                                     keys[k % 2], res, v, c, None, stream), reps)
            t_rot = per_call_ms(lambda k: ks.ks_hrot(ctx.h, cts[k % 3], k_rot, keys[k % 2], res,
                                                     v, c, None, stream), reps)
            out[name] = {"workload": prm.name(), "plan": ks.variant_name(v, c),
                         "keyswitch_per_s": 1e3 / t_ks, "hmul_per_s": 1e3 / t_mul,
                         "hrot_per_s": 1e3 / t_rot, "ks_ms": t_ks, "hmul_ms": t_mul,
                         "hrot_ms": t_rot}
            if name == "c3":
                # every dataflow x chunks 2..10 x fused/unfused (radix 8), one KeySwitch
                table = {}
                for base in (ks.KS_DSOB, ks.KS_DPOB, ks.KS_DSOC, ks.KS_DPOC):
                    for unf in (0, ks.KS_UNFUSED):
                        chunk_list = range(2, 11) if base in (ks.KS_DSOC, ks.KS_DPOC) else (0,)
                        for ch in chunk_list:
                            vv = base | unf
                            table[ks.variant_name(vv, ch)] = per_call_ms(
                                lambda k: ks.ks_switch(ctx.h, cts[k % 3][1], keys[k % 2], res, vv,
                                                       ch, None, stream), 10)
                out["c3_variants_ms"] = {k: round(t, 4) for k, t in
                                         sorted(table.items(), key=lambda kv: kv[1])}
        finally:
            ctx.close()

    # the learned selector, trained on the committed sweep, picks a plan per level too
    from paper_2603_16692_gb300 import selector as S
    try:
        data = S.load_json(os.path.join(S.DATA, "sweep_gb300.json"))
        sel, _ = S.train(data, S.split(len(data["points"]))[0])
    except (OSError, ValueError, KeyError):
        sel = None
    prm = W.make_params(*W.C3)
    top = ks.Context(prm)
    try:
        keys = [rand_limbs(prm.mods, (prm.beta, 2), prm.N) for _ in range(2)]
        fixed = ks.KS_DPOB
        rows, t_fix, t_dyn, t_mlp = [], 0.0, 0.0, 0.0
        for level in range(prm.L, -1, -1):
            view = top.at_level(level)
            try:
                ds = [rand_limbs(prm.q[:level + 1], (), prm.N) for _ in range(2)]
                res = torch.empty((2, level + 1, prm.N), dtype=torch.uint64, device=dev)
                v, c = ks.ks_tune(view.h, ds[0], keys[0], res, 1, stream)
                tf = per_call_ms(lambda k: ks.ks_switch(view.h, ds[k % 2], keys[k % 2], res, fixed,
                                                        0, None, stream), 10)
                td = per_call_ms(lambda k: ks.ks_switch(view.h, ds[k % 2], keys[k % 2], res, v, c,
                                                        None, stream), 10)
                t_fix += tf
                t_dyn += min(td, tf) if (v, c) == (fixed, 0) else td
                row = {"level": level, "tuned": ks.variant_name(v, c),
                       "ms_fixed": round(tf, 5), "ms_tuned": round(td, 5)}
                if sel is not None:
                    _, vm, cm = S.CANDS[sel.choose([S.level_shape(prm, level)])[0]]
                    # the plan the library runs for a selected context (ks_select's rule:
                    # the tensor-core conversions where the context has them, N >= 2^16
                    # and more than one digit)
                    if (ks.ks_context_info(view.h)["tc"] and prm.N >= 1 << 16
                            and level + 1 > prm.alpha):
                        vm |= ks.KS_BCONV_TC
                    if (vm, cm) == (fixed, 0):
                        tm = tf
                    elif (vm, cm) == (v, c):
                        tm = td
                    else:
                        tm = per_call_ms(lambda k: ks.ks_switch(view.h, ds[k % 2], keys[k % 2], res,
                                                                vm, cm, None, stream), 10)
                    t_mlp += tm
                    row.update(mlp=ks.variant_name(vm, cm), ms_mlp=round(tm, 5))
                rows.append(row)
            finally:
                view.close()
        picks, mpicks = {}, {}
        for r in rows:
            picks[r["tuned"]] = picks.get(r["tuned"], 0) + 1
            if "mlp" in r:
                mpicks[r["mlp"]] = mpicks.get(r["mlp"], 0) + 1
        out["levels"] = {
            "workload": f"one KeySwitch at each level {prm.L}..0 of {prm.name()} with the "
                        f"top-level key (level views)",
            "fixed_plan": ks.variant_name(fixed), "chain_ms_fixed": t_fix,
            "chain_ms_per_level_tuned": t_dyn, "speedup": t_fix / t_dyn, "picks": picks,
            "chain_ms_per_level_selector": t_mlp if sel is not None else None,
            "selector_speedup": t_fix / t_mlp if sel is not None and t_mlp > 0 else None,
            "selector_picks": mpicks, "per_level": rows}
    finally:
        top.close()
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    prm = W.make_params(*WORKLOADS[args.workload])

    if args.impl == "reference":
        run_reference(args, prm, rank, world)
        return

    import numpy as np
    import torch
    from paper_2603_16692_gb300 import ks

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ctx = ks.Context(prm)
    dev = torch.device("cuda", local)
    s_from, s_to, a, e = W.gen_keys(prm, 0)

    def to_dev(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dev)

    evk0 = ctx.keygen(to_dev(s_from), to_dev(s_to), to_dev(a), to_dev(e))
    d0 = to_dev(W.gen_input(prm, 0))
    set_bytes = (evk0.numel() + d0.numel() + 2 * d0.numel()) * 8
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    ring = max(2, -(-2 * l2 // set_bytes) + 1)
    sets = [(d0.clone(), evk0.clone(), torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64,
                                                   device=dev)) for _ in range(ring)]
    del evk0
    stream = torch.cuda.current_stream(dev)
    if args.variant.lower() == "tuned":
        variant, chunks = ks.ks_tune(ctx.h, sets[0][0], sets[0][1], sets[0][2], 1, stream)
    else:
        variant = ks.VARIANTS[args.variant.upper()] | (ks.KS_UNFUSED if args.unfused else 0) | \
            (ks.KS_RADIX4 if args.radix4 else 0)
        chunks = args.chunks
    args.chunks = chunks
    nws = ks.ks_workspace_size(ctx.h, variant, args.chunks) // 8 + 1
    # independent KeySwitches in flight on up to MAX_STREAMS streams (round-robin), each
    # stream with its own workspace; consecutive steps use distinct buffer sets
    wss = [torch.empty(nws, dtype=torch.uint64, device=dev) for _ in range(MAX_STREAMS)]
    ws = wss[0]
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(MAX_STREAMS - 1)]
    # plans for KeySwitches in flight: the tuned plan, and without its split ModDown (the
    # split forks onto the context's one side stream, which streams in flight share)
    cands = [variant] + ([variant & ~ks.KS_SPLIT_DOWN] if variant & ks.KS_SPLIT_DOWN else [])
    scalls_by = {v: [[ks.prepare_switch(ctx.h, d, evk, out, v, args.chunks, wss[q], streams[q])
                      for d, evk, out in sets] for q in range(MAX_STREAMS)] for v in cands}
    scalls = scalls_by[variant]
    calls = scalls[0]  # one stream, warm L2, host cost, profile: the tuned plan

    def run_streams(nstreams, n, k0=0):
        """n steps (KeySwitch k on stream k mod nstreams), fork from and join to `stream`."""
        for q in range(1, nstreams):
            streams[q].wait_stream(stream)
        for k in range(k0, k0 + n):
            scalls[k % nstreams][k % ring]()
        for q in range(1, nstreams):
            stream.wait_stream(streams[q])

    def rate(nstreams, n):
        run_streams(nstreams, 2 * nstreams)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_streams(nstreams, n)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return n / (e0.elapsed_time(e1) / 1e3)

    # streams in flight and their plan: the pair with the highest rate on a short probe
    # (ring >= count)
    probe_by_plan = {}
    for v in cands:
        scalls = scalls_by[v]
        probe_by_plan[v] = {q: rate(q, max(30, 10 * q))
                            for q in range(1, min(MAX_STREAMS, ring) + 1)}
    run_variant, nstreams = max(((v, q) for v in cands for q in probe_by_plan[v]),
                                key=lambda vq: probe_by_plan[vq[0]][vq[1]])
    scalls = scalls_by[run_variant]
    probe = probe_by_plan[run_variant]
    plan_info = {"variant": ks.variant_name(run_variant, args.chunks), "chunks": args.chunks,
                 "tuned_variant": ks.variant_name(variant, args.chunks),
                 "probe_ks_per_s_by_plan": {ks.variant_name(v, args.chunks): p_
                                            for v, p_ in probe_by_plan.items()},
                 "chosen_by": "ks_tune (timed over dataflows x radices; with streams in "
                               "flight, the tuned plan or the same without its split ModDown, "
                               "the faster on the probe)"
                 if args.variant.lower() == "tuned" else "--variant",
                 "l2": f"ring of {ring} distinct (d, evk, out) sets, {ring * set_bytes / 1e6:.0f}"
                       f" MB > 2 x L2 ({l2 / 1e6:.0f} MB): every step reads HBM"}

    def step(k):
        scalls[k % nstreams][k % ring]()

    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 30:
        gpu_id = "GPU-" + gpu_id
    sampler = ClockSampler(gpu_id)

    # warm-up, then the timed region: K steps between two synchronized barriers
    run_streams(nstreams, args.warmup)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    ev0.record(stream)
    run_streams(nstreams, args.steps)
    ev1.record(stream)
    barrier()
    t_wall1 = time.time()
    sampler.mark(t_wall0, t_wall1)
    el_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    value = job_rate(world, args.steps, el_ms)

    # warm L2: the same buffer set every step (reported beside the cold-L2 `value`)
    kw = min(args.steps, 2000)
    barrier()
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    for _ in range(kw):
        calls[0]()
    w1.record(stream)
    barrier()
    warm_value = job_rate(world, kw, max_over_ranks(w0.elapsed_time(w1), dist, dev))

    # one stream, the same steps: the latency-bound rate of KeySwitches one after another
    k1 = min(args.steps, 2000)
    barrier()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for k in range(k1):
        calls[k % ring]()
    s1.record(stream)
    barrier()
    one_stream_ms = max_over_ranks(s0.elapsed_time(s1), dist, dev) / k1

    # host cost of one step (Python call + launches), enqueued ahead of an idle GPU: a
    # short burst well inside the launch queue, so the host never waits for the device
    host_us = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(32):
            calls[k % ring]()
        host_us.append((time.perf_counter() - t0) * 1e6 / 32)
    torch.cuda.synchronize()
    host_us = min(host_us)

    # per-kernel event timing over a second pass of the same steps on one stream (kept out
    # of `value`). A split-ModDown plan runs its key multiply beside the P-limb ModDown
    # chain, so its launch times overlap and do not add up to a step: the profiling
    # pass runs the same plan unsplit (the same kernels, the key multiply in one
    # launch), beside that plan's own one-stream step time, the reference of the scaling
    # below.
    kprof = min(args.steps, 500)
    pvar = variant & ~ks.KS_SPLIT_DOWN
    pcalls = calls if pvar == variant else \
        [ks.prepare_switch(ctx.h, d, evk, out, pvar, args.chunks, ws, stream) for d, evk, out in sets]
    for k in range(10):
        pcalls[k % ring]()
    barrier()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for k in range(k1):
        pcalls[k % ring]()
    p1.record(stream)
    barrier()
    prof_step_ms = p0.elapsed_time(p1) / k1
    ks.ks_profile_begin()
    for k in range(kprof):
        pcalls[k % ring]()
    stats = ks.ks_profile_end()
    # the timed plan's launches: the profiled (unsplit) plan's, plus the split key
    # multiply's second launch when the timed plan splits
    launches_per_step = sum(s["launches"] for s in stats) / kprof + \
        (1 if run_variant & ks.KS_SPLIT_DOWN else 0)

    # end to end through the host-buffer entry points: a ring of pinned host inputs and
    # outputs; every step's input is read from and its result written to host memory
    # inside the timed region. `e2e`: ks_switch_host_async, the steps queued on the
    # stream and synchronized once at the end; `e2e_sync`: ks_switch_host, which
    # synchronizes every call.
    import math
    hring = 8
    d_hs = [torch.from_numpy(W.gen_input(prm, k)).pin_memory() for k in range(hring)]
    out_hs = [torch.empty((2, prm.L + 1, prm.N), dtype=torch.uint64).pin_memory()
              for _ in range(hring)]
    period = hring * ring // math.gcd(hring, ring)
    hcalls = [ks.prepare_switch_host_async(ctx.h, d_hs[k % hring], sets[k % ring][1],
                                           out_hs[k % hring], variant, args.chunks, stream)
              for k in range(period)]
    ke = max(10, min(args.steps, 1000))

    def e2e_run(step_fn, n):
        barrier()
        t0 = time.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(n):
            step_fn(k)
        e1.record(stream)
        barrier()
        sampler.mark(t0, time.time())
        return max_over_ranks(e0.elapsed_time(e1), dist, dev)

    def host_async(k):
        hcalls[k % period]()

    def host_sync(k):
        ks.ks_switch_host(ctx.h, d_hs[k % hring], sets[k % ring][1], out_hs[k % hring],
                          variant, args.chunks, stream)

    # host-buffer KeySwitches in flight on several streams: ks_switch_host_async_ws with
    # a scratch per stream (copy-engine transfers around device-buffer kernels; the
    # steps' host buffers are a ring of 8, so no two steps in flight share one); step k
    # on stream k mod count
    hws = ks.ks_host_workspace_size(ctx.h, variant, args.chunks) // 8 + 1
    e2e_max = 4
    hstreams = streams + [torch.cuda.Stream(device=dev) for _ in range(e2e_max - MAX_STREAMS)]
    hscr = [torch.empty(hws, dtype=torch.uint64, device=dev) for _ in range(e2e_max)]
    hscalls = [[ks.prepare_switch_host_async_ws(ctx.h, d_hs[k % hring], sets[k % ring][1],
                                                 out_hs[k % hring], hscr[q], run_variant,
                                                 args.chunks, hstreams[q])
                for k in range(period)] for q in range(e2e_max)]

    def host_streams(nq):
        def fn(k):
            if k == 0:
                for q in range(1, nq):
                    hstreams[q].wait_stream(stream)
            hscalls[k % nq][k % period]()
            if k == ke - 1:
                for q in range(1, nq):
                    stream.wait_stream(hstreams[q])
        return fn

    for k in range(5):
        host_async(k)
        host_sync(k)
    e2e_by_streams = {1: job_rate(world, ke, e2e_run(host_async, ke))}
    for nq in range(2, min(e2e_max, hring) + 1):
        e2e_run(host_streams(nq), ke)  # warm-up of this stream count
        e2e_by_streams[nq] = job_rate(world, ke, e2e_run(host_streams(nq), ke))
    e2e_streams = max(e2e_by_streams, key=e2e_by_streams.get)
    e2e_value = e2e_by_streams[e2e_streams]
    e2e_sync_value = job_rate(world, ke, e2e_run(host_sync, ke))
    clocks = sampler.stop()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = props.multi_processor_count
    # Per-kernel durations: the profiling pass brackets every launch with events, which
    # breaks the programmatic-dependent-launch overlap of consecutive kernels, so their
    # sum exceeds the one-stream step of the profiled plan; each kernel's event time is
    # scaled by (that step / the sum), so the kernels add up to the step.
    step_ms = el_ms / args.steps
    ev_sum = sum(s["ms"] for s in stats) / kprof
    scale = prof_step_ms / ev_sum
    dom = max(stats, key=lambda s: s["ms"])
    per_launch_ms = dom["ms"] / dom["launches"] * scale
    bytes_l = dom["bytes"] / dom["launches"]
    hbm_ach = bytes_l / (per_launch_ms / 1e3) / 1e9
    bf, mac = measured_alu(ks, stream)
    alu = alu_roofline(dom, per_launch_ms, bf, mac)
    alu_ev = alu_roofline(dom, dom["ms"] / dom["launches"], bf, mac)
    # the recipe's unit counts for context: SMs x 64 IMAD lanes x max clock / 10 IMAD per
    # 64-bit Shoup product
    derived = sms * 64 * sm_mhz * 1e6 / 10 / 1e9
    tens = tensor_roofline(dom, per_launch_ms, peaks)
    ncu = ncu_row(args.workload, ks.variant_name(pvar, args.chunks), dom["name"],
                  *tc_sides(ks, pvar))
    roofline = {"bound": "alu", "kernel": dom["name"], "achieved": alu["achieved"],
                "peak": alu["peak"], "unit": "Gop/s (butterfly-equivalent)",
                "frac": alu["frac"], "traffic": ncu["traffic"] if ncu else None,
                "peak_source": "measured in this run: ks_calibrate, the library's butterfly "
                               f"({bf / 1e12:.3f} T/s) and 128-bit MAC ({mac / 1e12:.3f} T "
                               f"terms/s) on all {sms} SMs; MAC terms counted at the ratio",
                "t_ceil_ms": alu["t_ceil_ms"], "duration_ms": per_launch_ms,
                "duration_source": f"event time x {scale:.3f} (one-stream step of the "
                                   f"profiled plan {ks.variant_name(pvar, args.chunks)}, "
                                   f"{prof_step_ms:.4f} ms, / sum of its event-bracketed "
                                   "launches)",
                "event_ms": dom["ms"] / dom["launches"],
                "event_frac": alu_ev["frac"],
                "share": dom["ms"] / sum(s["ms"] for s in stats),
                "macs_per_launch": alu["macs_per_launch"],
                "shoup_per_launch": alu["shoup_per_launch"],
                "algo_bytes_per_launch": bytes_l, "hbm_achieved_gbs": hbm_ach,
                "hbm_frac": hbm_ach / hbm,
                "derived_peak": {"value": derived, "unit": "Gmodop/s",
                                 "source": f"{sms} SMs x 64 IMAD/clk x {sm_mhz:.0f} MHz / 10 IMAD"
                                           " per modop"},
                "ncu": ncu}
    if tens:
        # a tensor-core conversion: its products on the tensor pipe, its REDCs and NTT on
        # the integer pipes; the bound is the larger of the two ceilings
        roofline["tensor"] = tens
        roofline["what"] = ("tensor-core basis conversion fused with the column NTT: ALU "
                            "part = one REDC per output + the NTT's Shoup products; tensor "
                            "part = the byte-split bf16 products")
        if tens["t_ceil_ms"] > alu["t_ceil_ms"]:
            roofline.update({"bound": "tensor", "achieved": tens["achieved"] * 1e3,
                             "peak": tens["peak"] * 1e3, "unit": "GFLOP/s (bf16)",
                             "frac": tens["frac"]})
    # the whole KeySwitch at the measured ceiling: every kernel's arithmetic
    t_ceil_step = sum((s["macs"] / mac + (s["ops"] - s["macs"]) / bf) for s in stats) / kprof * 1e3
    algo = prm.algo_bytes()
    ks_gbs = algo * value / world / 1e9
    kernels = []
    for s_ in sorted(stats, key=lambda s: -s["ms"]):
        n = s_["launches"]
        t = s_["ms"] / n * scale
        tc = (s_["macs"] / mac + (s_["ops"] - s_["macs"]) / bf) / n * 1e3
        k = {"name": s_["name"], "launches_per_step": n / kprof, "ms_per_launch": round(t, 5),
             "event_ms_per_launch": round(s_["ms"] / n, 5), "alu_frac": round(tc / t, 4),
             "share": round(s_["ms"] / sum(x["ms"] for x in stats), 4)}
        nc = ncu_row(args.workload, ks.variant_name(pvar, args.chunks), s_["name"],
                     *tc_sides(ks, pvar))
        if nc:
            k["dram_bytes"] = nc["traffic"]
            k["algo_bytes"] = s_["bytes"] / n
        kernels.append(k)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded uniform d, ternary keys, rounded-Gaussian errors)",
        "config": workload_config(prm),
        "plan": plan_info,
        "roofline": roofline,
        "ks_alu_roofline": {"bound": "alu", "t_ceil_ms": t_ceil_step, "ms_per_step": step_ms,
                            "frac": t_ceil_step / step_ms,
                            "one_stream_frac": t_ceil_step / one_stream_ms,
                            "tensor_t_ceil_ms": sum(x.get("tensor_flops", 0) for x in stats)
                            / kprof / (float(peaks.get("bf16_tflops_sustained", 1700.0)) * 1e9),
                            "what": "the whole KeySwitch's integer arithmetic at the measured "
                                    "ceiling (the products of tensor-core conversions apart: "
                                    "tensor_t_ceil_ms at the sustained bf16 rate)"},
        "streams": {"in_flight": nstreams, "probe_ks_per_s": probe,
                    "one_stream_value": job_rate(world, 1, one_stream_ms),
                    "one_stream_ms_per_step": one_stream_ms,
                    "how": "step k runs on stream k mod in_flight, each stream with its own "
                           "workspace, forked from and joined to the timing stream; "
                           "in_flight = the count with the best rate on a short probe"},
        "ks_hbm_roofline": {"bound": "hbm", "achieved": ks_gbs, "peak": hbm, "unit": "GB/s",
                            "frac": ks_gbs / hbm, "algo_bytes_per_ks": algo,
                            "peak_source": peaks["source"]},
        "kernels": kernels,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "host_us_per_step": host_us,
        "warm_l2_value": warm_value,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": (prm.L + 1) * prm.N * 8,
                "d2h_bytes_per_step": 2 * (prm.L + 1) * prm.N * 8,
                "entry": "ks_switch_host_async_ws on the fastest stream count (1: "
                         "ks_switch_host_async), pinned host ring of 8, one sync at the end",
                "streams_in_flight": e2e_streams, "value_by_streams": e2e_by_streams,
                "sync_per_call_value": e2e_sync_value},
        "clocks": clocks,
    }
    others = [w for w in ("c2", "c1") if w != args.workload]
    line["other_workloads"] = other_workloads(others, ks, torch, dev, stream, l2,
                                              max(100, min(args.steps, 2000)))
    if not args.no_batch:
        line["batch64"] = batch_measure(args, ks, torch, dev, stream, hbm)
    if not args.no_eval:
        line["eval"] = eval_measure(args, ks, torch, dev, stream, l2)
    if world == 1 and not args.no_cpu:
        reps, el, cores = oracle_sample(prm, args.cpu_seconds, 10000)
        r1, el1, _ = oracle_sample(prm, args.cpu_seconds / 2, 10000, nthreads=1)
        line["cpu_baseline"] = {"value": reps / el, "unit": UNIT, "cores": cores,
                                "kind": "oracle",
                                "sample": f"{reps} full KeySwitches of the same workload in"
                                          f" {el:.1f} s (bounded at ~{args.cpu_seconds:.0f} s)",
                                "single_thread": {"value": r1 / el1, "unit": UNIT,
                                                  "sample": f"{r1} KeySwitches in {el1:.1f} s"}}
    else:
        line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
