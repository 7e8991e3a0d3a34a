"""C(m) curves of four probe kernels on this GPU, measured with the blocker
method of §3 (Fig. 1), their least-squares fit C(m) = a / m + b (§3.3's model
without interference), and the interference factor k = C_interfered(m) / C(m)
with the SMs not given to the kernel streaming HBM (§3.3's memory-intensive
co-runner).  Everything runs through gpa_measure_wcet / gpa_fit_wcet.

    python -m paper_2105_10312_gb300.measure [--reps 5] [--kernels VADD,COMPUTE] [--out curves.json]

In the task model of the library (times in microseconds, k per mille), a
kernel whose fit is (a, b) in milliseconds has A = 10^6 a and B = 10^6 b:
C(m) = k (A + B m) / (10^6 m) microseconds.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

SIZES = {"VADD": 1 << 25, "TRANSPOSE": 8192, "STENCIL": 8192, "COMPUTE": 1 << 24}
M_LIST = (1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 76, 96, 114, 128, 152)


def run(reps=5, device=0, kernels=None, m=None, sizes=None):
    import torch

    import paper_2105_10312_gb300 as gpa
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    ms_list = sorted({x for x in (m or M_LIST) if 1 <= x <= sms} | {sms})
    kernels = list(kernels or SIZES)
    sizes = dict(SIZES, **(sizes or {}))
    ctx = gpa.Context(device)
    out = {"sm_count": sms, "m": ms_list, "reps": reps, "kernels": {}}
    try:
        for k in kernels:
            alone, used = gpa.measure_wcet(ctx, k, ms_list, sizes[k], reps=reps)
            inter, used_i = gpa.measure_wcet(ctx, k, ms_list, sizes[k], reps=reps, interfere=True)
            a, b = gpa.fit_wcet(ms_list, alone)
            mm = np.array(ms_list, np.float64)
            fit = a / mm + b
            ok = alone > 0
            rel = np.abs(fit[ok] - alone[ok]) / alone[ok]
            ratio = [float(i / x) for i, x, q in zip(inter, alone, ms_list) if q < sms and i > 0 and x > 0]
            kf = float(np.median(ratio)) if ratio else None
            out["kernels"][k] = {
                "n": sizes[k], "ms": alone.tolist(), "sms_used": used.tolist(),
                "ms_interfered": inter.tolist(), "sms_used_interfered": used_i.tolist(),
                "a_ms": a, "b_ms": b, "A": int(round(1e6 * a)), "B": int(round(1e6 * b)),
                "fit_max_rel_err": float(rel.max()) if rel.size else None,
                "k": kf, "k_pm": int(round(1000 * kf)) if kf else None,
            }
    finally:
        ctx.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--kernels", default=",".join(SIZES))
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    res = run(args.reps, kernels=[k.strip().upper() for k in args.kernels.split(",") if k.strip()])
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f)
    print("m         " + " ".join(f"{x:7d}" for x in res["m"]))
    for k, r in res["kernels"].items():
        print(f"{k:9s} " + " ".join(f"{t:7.3f}" for t in r["ms"]) + "  ms alone")
        print(f"{'':9s} " + " ".join(f"{t:7.3f}" for t in r["ms_interfered"]) + "  ms with HBM co-runner")
        print(f"{'':9s} a = {r['a_ms']:.4f} ms, b = {r['b_ms']:.4f} ms (max rel. fit error "
              f"{r['fit_max_rel_err']:.2f}); k = {r['k']}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
