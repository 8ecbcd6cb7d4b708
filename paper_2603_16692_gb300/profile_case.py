"""One KeySwitch (or HMUL / HROT) of a given (dnum, N, L) and plan, for profilers.

Sets up a context and seeded random operands (uniform residues; no key generation,
so that the only library kernels the process launches are the ones of the single
timed operation), then runs the operation once (``--reps`` times) and exits. The
kernel names all start with ``k_``, so ``ncu -k regex:^k_`` captures exactly the
operation's launches.

    python -m paper_2603_16692_gb300.profile_case --cfg 4,16,30 --variant DPOB

With ``--stats`` (not for profilers: it adds timing and calibration launches) it also
prints, per kernel, the event time of a launch and its fraction of the measured
ceiling of its own arithmetic (``ks_calibrate``), and the same for the whole operation.
"""
from __future__ import annotations

import argparse

from . import ks
from . import workload as W


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--cfg", default="4,16,30", help="dnum,log2N,L")
    ap.add_argument("--variant", default="DPOB", help="DSOB / DPOB / DSOC / DPOC")
    ap.add_argument("--chunks", type=int, default=0)
    ap.add_argument("--unfused", action="store_true")
    ap.add_argument("--radix", type=int, default=8, choices=[4, 8, 16])
    ap.add_argument("--sched", default="",
                    help="per-stage radix and column tile, e.g. km4,dnr16,colalt-inv "
                         "(stages inv, upc, km, dnc, dnr), split, tc; 'tuned' = ks_tune's "
                         "choice")
    ap.add_argument("--op", default="switch", choices=["switch", "hmul", "hrot"])
    ap.add_argument("--level", type=int, default=-1, help="run on a level view (default: top)")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--stats", action="store_true",
                    help="print per-kernel time and fraction of the measured ALU ceiling")
    args = ap.parse_args(argv)

    import torch
    dnum, logn, L = (int(x) for x in args.cfg.split(","))
    prm = W.make_params(dnum, logn, L)
    dev = torch.device("cuda", 0)
    v = ks.VARIANTS[args.variant.upper()] | (ks.KS_UNFUSED if args.unfused else 0) | \
        {4: ks.KS_RADIX4, 8: 0, 16: ks.KS_RADIX16}[args.radix] | parse_sched(args.sched)
    top = ks.Context(prm)
    ctx = top.at_level(args.level) if args.level >= 0 else top
    nq = ctx.nq
    g = W.rng(2024, 11)
    evk = torch.from_numpy(W.uniform_limbs(g, prm.mods * (2 * prm.beta), prm.N).reshape(
        prm.beta, 2, prm.QP, prm.N)).to(dev)
    ct = torch.from_numpy(W.uniform_limbs(g, prm.q[:nq] * 2, prm.N).reshape(2, nq, prm.N)).to(dev)
    ct2 = torch.from_numpy(W.uniform_limbs(g, prm.q[:nq] * 2, prm.N).reshape(2, nq, prm.N)).to(dev)
    out = torch.empty_like(ct)
    torch.cuda.synchronize()
    if args.sched == "tuned":
        v, args.chunks = ks.ks_tune(ctx.h, ct[1].contiguous(), evk, out, 1)

    def run():
        if args.op == "switch":
            ctx.switch(ct[1], evk, out, v, args.chunks)
        elif args.op == "hmul":
            ctx.hmul(ct, ct2, evk, out, v, args.chunks)
        else:
            ctx.hrot(ct, ks.galois_elt(1, prm.N), evk, out, v, args.chunks)

    for _ in range(args.reps):
        run()
    torch.cuda.synchronize()
    print(f"{args.op} {prm.name()} level {nq - 1} {ks.variant_name(v, args.chunks)}: ok")
    if args.stats:
        stats(run, max(args.reps, 20))
    if ctx is not top:
        ctx.close()
    top.close()


def parse_sched(text: str) -> int:
    """'km4,dnr16,colalt' -> KS_STAGE_RADIX(KS_ST_KM, KS_R4) | ... | KS_COLTILE_ALT."""
    v = 0
    for item in filter(None, text.split(",")):
        if item == "split":
            v |= ks.KS_SPLIT_DOWN
        elif item == "tc":
            v |= ks.KS_BCONV_TC
        elif item == "tcdown":
            v |= ks.KS_BCONV_TC_DOWN
        elif item == "colalt":
            v |= ks.KS_COLTILE_ALT
        elif item.startswith("colalt-"):
            v |= {"inv": ks.KS_COLALT_INV, "upc": ks.KS_COLALT_UPC,
                  "dnc": ks.KS_COLALT_DNC}[item[len("colalt-"):]]
        elif item == "tuned":
            continue
        else:
            name = item.rstrip("0123456789")
            v |= ks.KS_STAGE_RADIX(ks.STAGE_NAMES.index(name),
                                   {4: ks.KS_R4, 8: ks.KS_R8, 16: ks.KS_R16}[int(item[len(name):])])
    return v


def stats(run, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    op_ms = e0.elapsed_time(e1) / reps
    ks.ks_profile_begin()
    for _ in range(reps):
        run()
    rows = ks.ks_profile_end()
    bf = max(ks.ks_calibrate(ks.KS_CAL_BUTTERFLY, 16384) for _ in range(3))
    mac = max(ks.ks_calibrate(ks.KS_CAL_MAC, 4096) for _ in range(3))
    print(f"measured ceiling: {bf / 1e12:.3f} T butterflies/s, {mac / 1e12:.3f} T MAC terms/s")
    print(f"{'kernel':22s} {'us/launch':>10s} {'ceil us':>8s} {'frac':>6s} {'share':>6s}")
    total = sum(r["ms"] for r in rows)
    ceil_op = 0.0
    for r in sorted(rows, key=lambda r: -r["ms"]):
        ceil = (r["macs"] / mac + (r["ops"] - r["macs"]) / bf) * 1e6 / r["launches"]
        us = r["ms"] * 1e3 / r["launches"]
        ceil_op += ceil * r["launches"] / reps
        tc = r.get("tensor_flops", 0) / r["launches"]
        extra = f"  tensor {tc / (us * 1e-6) / 1e12:.0f} TFLOP/s" if tc else ""
        print(f"{r['name']:22s} {us:10.2f} {ceil:8.2f} {ceil / us:6.1%} {r['ms'] / total:6.1%}"
              + extra)
    print(f"operation: {op_ms * 1e3:.1f} us, integer arithmetic at the measured ceiling "
          f"{ceil_op:.1f} us ({ceil_op / (op_ms * 1e3):.1%})")


if __name__ == "__main__":
    main()
