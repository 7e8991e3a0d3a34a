"""Data of the paper's §7 experiments on synthetic task sets (Figs. 4-7):
per total utilisation U, the schedulability rate, the number of partitions
and the scheduled (inflated) workload against its bounds, for the 1G
baseline and the four heuristic variants SMS/BF x ACT/INA, computed on the
GPU through the library.

    python -m paper_2105_10312_gb300.figures [--tasks 50|200] [--sets-per-step 100] [--sched dm|edf]
                                             [--out figs.json]

The setting is §7's: 68 SMs, 50 tasks per set (Figs. 4 and 5) or 200 (Figs. 6
and 7), U = 2, 4, ..., 68, D = 0.75 T,
periods from the divisors of 4000 in [50, 4000], a 50 % memory-intensive
ratio, b = 0.02 a (compute) / 0.1 a (memory).  The workload bounds of §7's
efficiency figure are, per task set, Best = sum_i u_i (every task without
interference) and Worst = sum_i k_i u_i with the conflict factor of its type
(every task in conflict); a heuristic's scheduled load of a set it
allocates is W / 1000 = sum over its partitions of sum_i k_i(P) u_i.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

VARIANTS = (("1G", "ONE_GPU", False), ("SMS_ACT", "SMS", True), ("SMS_INA", "SMS", False),
            ("BF_ACT", "BF", True), ("BF_INA", "BF", False))


def workload_bounds(sets, k_c_pm, k_m_pm):
    """Best and Worst scheduled load of every set (units of U: u_ppm / 10^6)."""
    off = np.asarray(sets["set_off"], dtype=np.int64)
    u = np.asarray(sets["u_ppm"], dtype=np.float64)
    k = np.where(np.asarray(sets["type"]) == 1, k_m_pm, k_c_pm).astype(np.float64)
    best = np.add.reduceat(u, off[:-1]) if len(u) else np.zeros(len(off) - 1)
    worst = np.add.reduceat(k * u, off[:-1]) / 1000.0 if len(u) else np.zeros(len(off) - 1)
    empty = off[1:] == off[:-1]
    best[empty] = 0.0
    worst[empty] = 0.0
    return best / 1e6, worst / 1e6


def aggregate(results, best, worst, steps):
    """Per-step averages from per-set results.  results: name -> dict of
    per-set arrays (verdict, n_parts, W); set s belongs to step s % steps."""
    nsets = len(best)
    step = np.arange(nsets) % steps
    out = {"steps": steps, "best": [], "worst": [], "variants": {}}
    for j in range(steps):
        sel = step == j
        out["best"].append(float(best[sel].mean()) if sel.any() else None)
        out["worst"].append(float(worst[sel].mean()) if sel.any() else None)
    for name, r in results.items():
        v = np.asarray(r["verdict"]).astype(bool)
        parts = np.asarray(r["n_parts"], dtype=np.float64)
        load = np.asarray(r["W"], dtype=np.float64) / 1e9
        span = worst - best
        rel = np.where(span > 0, (load - best) / np.where(span > 0, span, 1.0), 0.0)
        rate, mparts, mload, mrel = [], [], [], []
        for j in range(steps):
            sel = step == j
            ok = sel & v
            rate.append(float(v[sel].mean()) if sel.any() else None)
            mparts.append(float(parts[ok].mean()) if ok.any() else None)
            mload.append(float(load[ok].mean()) if ok.any() else None)
            mrel.append(float(rel[ok].mean()) if ok.any() else None)
        out["variants"][name] = {"rate": rate, "parts": mparts, "load": mload, "load_in_bounds": mrel}
    return out


def run(sets_per_step=100, sched="DM", device=0, tasks=50):
    """Allocate the §7 batch of `tasks` (50 or 200) tasks per set with every
    variant on the GPU; returns the aggregate (see aggregate) plus the U of
    each step."""
    import torch

    import paper_2105_10312_gb300 as gpa
    from paper_2105_10312_gb300 import workloads as W
    name = {50: "paper50", 200: "paper200"}[tasks]
    p = W.gen_params(name, nsets=34 * sets_per_step)
    s = gpa.gen_tasksets(**p)
    md = W.model(name)
    d = gpa.to_device(s, f"cuda:{device}")
    stream = torch.cuda.Stream(device)
    ctx = gpa.Context(device, stream=stream)
    results = {}
    try:
        for name, policy, act in VARIANTS:
            out = ctx.allocate(d, **md, policy=policy, act=act, sched=sched)
            ctx.sync()
            results[name] = {k: out[k].cpu().numpy() for k in ("verdict", "n_parts", "W")}
    finally:
        ctx.close()
    best, worst = workload_bounds(s, md["k_c_pm"], md["k_m_pm"])
    agg = aggregate(results, best, worst, p["U_steps"])
    agg["U"] = [(p["U_lo_ppm"] + j * (p["U_hi_ppm"] - p["U_lo_ppm"]) // (p["U_steps"] - 1)) / 1e6
                for j in range(p["U_steps"])]
    agg["sets_per_step"] = sets_per_step
    agg["sched"] = sched
    agg["tasks"] = tasks
    return agg


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--tasks", type=int, choices=[50, 200], default=50)
    ap.add_argument("--sets-per-step", type=int, default=100)
    ap.add_argument("--sched", choices=["dm", "edf"], default="dm")
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    agg = run(args.sets_per_step, args.sched.upper(), tasks=args.tasks)
    text = json.dumps(agg)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print("U     " + " ".join(f"{u:5.0f}" for u in agg["U"]))
    for name, v in agg["variants"].items():
        print(f"{name:8s}" + " ".join("   - " if r is None else f"{r:5.2f}" for r in v["rate"]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
