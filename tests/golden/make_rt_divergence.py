"""Writes tests/golden/rt_divergence.json from the FP64 oracle alone.

The Rayleigh-Taylor configuration (256 x 1024, rho_A/rho_B = 3, W = 4,
sigma = 5e-5, sqrt(g L) = 0.04, Re = 3000, walls in y; the parameter
readings of workloads.rayleigh_taylor) run by the oracle for its stated
20,000 steps: it does not get there.  Recorded: max |u| and the totals
sum rho, sum phi every 1000 steps, and the first step after which the
oracle's fields are no longer finite.

    python tests/golden/make_rt_divergence.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1507_03521_gb300 import workloads as W  # noqa: E402


def main():
    p, phi = W.rayleigh_taylor()
    try:
        lib = oracle.build_omp()
        threads = oracle.set_threads(len(os.sched_getaffinity(0)), lib)
    except Exception:
        lib, threads = None, 1
    o = oracle.Oracle(p, lib=lib)
    o.init_phi(phi)
    m0, t0 = o.mass()
    every = []
    first_nonfinite = None
    while o.step_count < 20000:
        o.step(1000 if o.step_count % 1000 == 0 and o.step_count + 1000 <= 8000 else 1)
        f = o.fields()
        finite = all(np.isfinite(f[k]).all() for k in ("phi", "ux", "uy", "p"))
        if not finite:
            first_nonfinite = o.step_count
            break
        if o.step_count % 1000 == 0:
            m, t = o.mass()
            every.append({"step": o.step_count,
                          "umax": float(max(np.abs(f["ux"]).max(), np.abs(f["uy"]).max())),
                          "mass": m, "phi_total": t})
            print(every[-1], flush=True)
    out = {"source": "FP64 oracle (oracle/orc.c), OpenMP build, "
                     f"{threads} threads; workloads.rayleigh_taylor()",
           "config": "Rayleigh-Taylor 256 x 1024, 20,000 steps stated",
           "mass0": m0, "phi_total0": t0, "every_1000": every,
           "first_nonfinite_step": first_nonfinite}
    with open(os.path.join(HERE, "rt_divergence.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("first non-finite step:", first_nonfinite)


if __name__ == "__main__":
    main()
