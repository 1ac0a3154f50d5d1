"""Precision study of the storage forms on the 4096 x 4096 precision workload.

Runs the same seeded workload (512 droplets, rho_A/rho_B = 100, sigma =
1e-3, M = 0.05, tau = 0.8) in FP64, FP32, FP16-storage and BF16-storage on
the GPU and reports, every `--every` steps, each form's error against the
FP64 path (which the parity tests check against the FP64 oracle): max-abs
and RMS differences of phi, u and p, and the drift of the total mass sum
rho and of sum phi from their initial values.

    python precision_study.py --steps 10000 --every 1000

Prints one JSON object per checkpoint and a final summary line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    import torch

    from paper_1507_03521_gb300 import build, lbm
    from paper_1507_03521_gb300 import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--rho-ratio", type=float, default=100.0,
                    help="rho_A / rho_B (the workload's is 100)")
    args = ap.parse_args()
    build.build()
    n_drops = 512 if args.n == 4096 else max(1, int(512 * (args.n / 4096) ** 2))
    p, phi = W.precision(n=args.n, n_drops=n_drops)
    p = dict(p, rho_B=p["rho_A"] / args.rho_ratio)
    forms = ("f64", "f32", "f16s", "bf16s", "f16d", "bf16d")
    sims = {}
    m0 = {}
    for f in forms:
        s = lbm.Sim(p, f)
        s.init_phi(phi)
        sims[f] = s
        m0[f] = s.mass()
    t0 = time.time()
    done = 0
    rows = []
    while done < args.steps:
        k = min(args.every, args.steps - done)
        for s in sims.values():
            s.step(k)
        done += k
        ref = sims["f64"].fields(("phi", "ux", "uy", "p"))
        rec = {"step": done}
        for f in forms:
            try:
                m = sims[f].mass()
                drift = {"mass_rel": (m[0] - m0[f][0]) / m0[f][0], "phi_total_abs": m[1] - m0[f][1]}
            except lbm.LBMError as e:
                drift = {"error": str(e)}
            if f == "f64":
                rec[f] = {"drift": drift}
                continue
            cur = sims[f].fields(("phi", "ux", "uy", "p"))
            err = {}
            for key in ("phi", "ux", "uy", "p"):
                d = (cur[key].double() - ref[key]).abs()
                err[key] = {"max": float(d.max()), "rms": float(d.pow(2).mean().sqrt())}
            rec[f] = {"err_vs_f64": err, "drift": drift}
        rec["elapsed_s"] = round(time.time() - t0, 1)
        rows.append(rec)
        print(json.dumps(rec), flush=True)
    for s in sims.values():
        s.close()
    # the last checkpoint at which every form is still finite
    finite = [r for r in rows if all(np.isfinite(r[f]["err_vs_f64"]["phi"]["max"]) for f in forms[1:])]
    if not finite:
        print(json.dumps({"summary": "no finite checkpoint"}), flush=True)
        return 0
    last = finite[-1]
    summary = {"workload": f"precision-{args.n}x{args.n}-{n_drops}-droplets-rho{args.rho_ratio:g}",
               "steps": args.steps, "last_finite_step": last["step"],
               "phi_max_err": {f: last[f]["err_vs_f64"]["phi"]["max"] for f in forms[1:]},
               "u_max_err": {f: max(last[f]["err_vs_f64"]["ux"]["max"], last[f]["err_vs_f64"]["uy"]["max"])
                             for f in forms[1:]},
               "p_max_err": {f: last[f]["err_vs_f64"]["p"]["max"] for f in forms[1:]},
               "mass_drift_rel": {f: last[f]["drift"].get("mass_rel") for f in forms}}
    print(json.dumps({"summary": summary}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
