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
    o = fast_oracle(p)
    o.init_phi(pert, ux, uy)
    o.step(steps)
    f = o.fields()
    return {k: float(np.abs(f[k] - base[k]).max()) for k in base}


def check64(g, o, spread, tag, keys=FIELDS):
    for k in keys:
        tol = max(1e-12 * float(np.abs(o[k]).max()), 10.0 * spread[k])
        err = float(np.abs(g[k] - o[k]).max())
        assert err <= tol, f"{tag}: {k} error {err:.3e} > {tol:.3e}"




def fast_oracle(p):
    """The oracle, from its OpenMP build where the compiler has OpenMP (bit-
    identical to the serial build), else the serial build."""
    try:
        lib = oracle.build_omp()
    except Exception:
        return oracle.Oracle(p)
    import os
    oracle.set_threads(len(os.sched_getaffinity(0)), lib)
    return oracle.Oracle(p, lib=lib)


def linear_rate(p, phibar, a, b):
    """Growth rate per step of a small mode of wavenumbers (a, b) about a
    uniform phibar, from Eq. 19 linearised at u = 0:
        d phi^/dt = (1 + gamma phibar) lambda L (psi'' - kappa L) phi^,
    with L the symbol of the isotropic lattice Laplacian,
        L = (2/cs2) [(2/9)(cos a + cos b) + (1/9) cos a cos b - 5/9],
    psi'' the second derivative of the double well of Eq. 2 at phibar,
    kappa and beta from Eqs. 3-4 and gamma from Eq. 17 (lambda = M)."""
    import math
    pa, pb = p["phi_A"], p["phi_B"]
    d = pa - pb
    kappa = 3.0 * p["sigma"] * p["W"] / (2.0 * d * d)
    beta = 12.0 * p["sigma"] / (p["W"] * d ** 4)
    gamma = (p["rho_A"] - p["rho_B"]) / (p["rho_B"] * pa - p["rho_A"] * pb)
    mid = 0.5 * (pa + pb)
    # psi' = 4 beta (phi - pa)(phi - pb)(phi - mid)
    psi2 = 4.0 * beta * ((phibar - pb) * (phibar - mid) + (phibar - pa) * (phibar - mid)
                         + (phibar - pa) * (phibar - pb))
    L = 6.0 * ((2.0 / 9.0) * (math.cos(a) + math.cos(b)) + (1.0 / 9.0) * math.cos(a) * math.cos(b)
               - 5.0 / 9.0)
    return (1.0 + gamma * phibar) * p["M"] * L * (psi2 - kappa * L)


def mode_amplitude(phi, mode):
    """Projection of phi - mean on a sin*cos mode (normalised: amplitude)."""
    return float(np.sum((phi - phi.mean()) * mode) / np.sum(mode * mode))
