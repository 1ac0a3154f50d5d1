"""Shared helpers of the GPU parity tests (the FP64 comparison bar)."""
import numpy as np

import oracle

FIELDS = ("phi", "rho", "p", "ux", "uy", "mu")


# FP64 bar: max |gpu - oracle| <= max(1e-12 max |oracle|, 10 s), where s is
# the change of the oracle's own field when each phi0 value is moved by one
# ulp: the conditioning of the problem under roundoff.  The GPU evaluates
# the same formulas in a different order, i.e. with different roundoff at
# every step; for phi, rho, p and mu the 1e-12 term governs, while a small
# velocity formed from cancelling terms can move by more than 1e-12 of its
# maximum from input roundoff alone.
def oracle_spread(p, phi, ux, uy, steps, base):
    rng = np.random.default_rng(12345)
    pert = np.where(rng.uniform(size=phi.shape) < 0.5, np.nextafter(phi, np.inf),
                    np.nextafter(phi, -np.inf))
    o = oracle.Oracle(p)
    o.init_phi(pert, ux, uy)
    o.step(steps)
    f = o.fields()
    return {k: float(np.abs(f[k] - base[k]).max()) for k in base}


def check64(g, o, spread, tag, keys=FIELDS):
    for k in keys:
        tol = max(1e-12 * float(np.abs(o[k]).max()), 10.0 * spread[k])
        err = float(np.abs(g[k] - o[k]).max())
        assert err <= tol, f"{tag}: {k} error {err:.3e} > {tol:.3e}"


