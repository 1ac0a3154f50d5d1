"""Shared helpers of the GPU parity tests (the FP64 comparison bar)."""
import numpy as np

import oracle

FIELDS = ("phi", "rho", "p", "ux", "uy", "mu")


# FP64 bar (Sec. 3, Eqs. 30-32 define the fields compared).
#   phi, rho, p, mu:  max |gpu - oracle| <= 1e-12 max |oracle|.
#   ux, uy:           max |gpu - oracle| <= max(1e-12 max |oracle|, 10 s),
# where s is the change of the oracle's own velocity field when each phi0
# value is moved by one ulp: the conditioning of the problem under
# roundoff.  The GPU evaluates the same formulas in a different order, i.e.
# with different roundoff at every step.  A small velocity formed from
# cancelling terms (a relaxing flat layer, |u_y| <= 3e-5) moves by more than
# 1e-12 of its maximum under input roundoff alone, so only the velocities
# get the conditioning term; phi, rho, p and mu are held to the plain
# relative bound.
SPREAD_FIELDS = ("ux", "uy")
PARITY_LOG = []  # (tag, field, error, bar, governing term) of every check


def oracle_spread(p, phi, ux, uy, steps, base):
    rng = np.random.default_rng(12345)
    pert = np.where(rng.uniform(size=phi.shape) < 0.5, np.nextafter(phi, np.inf),
                    np.nextafter(phi, -np.inf))
    o = fast_oracle(p)
    o.init_phi(pert, ux, uy)
    o.step(steps)
    f = o.fields()
    return {k: float(np.abs(f[k] - base[k]).max()) for k in base}


def bar64(k, o, spread, rel=1e-12):
    """The FP64 bar of field k and the term that sets it."""
    rel_term = rel * float(np.abs(o[k]).max())
    if k in SPREAD_FIELDS and spread is not None and 10.0 * spread[k] > rel_term:
        return 10.0 * spread[k], "10s"
    return rel_term, "rel"


def check64(g, o, spread, tag, keys=FIELDS, rel=1e-12):
    for k in keys:
        tol, term = bar64(k, o, spread, rel)
        err = float(np.abs(g[k] - o[k]).max())
        PARITY_LOG.append((tag, k, err, tol, term))
        print(f"PARITY64 {tag} {k} err={err:.3e} bar={tol:.3e} term={term} "
              f"ratio={err / tol if tol > 0 else float('inf'):.3f}")
        assert err <= tol, f"{tag}: {k} error {err:.3e} > {tol:.3e} ({term})"


# Long-run FP64 bar (runs of hundreds to thousands of steps).  Two rounding
# orders drift apart step by step: the GPU's roundoff differs from the
# oracle's by about an ulp in every population at every step, and the run
# carries each step's difference forward.  So the relative term is taken
# per 100 steps (worst case linear growth), and every field may also use
# the conditioning term 10 s, where s is measured on the oracle itself over
# the same run with that very perturbation: every population moved by one
# ulp, in a seeded random direction, before every step (oracle_jitter_spread):
#   max |gpu - oracle| <= max(1e-12 (steps / 100) max |oracle|, 10 s).
# An unstable set-up (spinodal decomposition, a Rayleigh-Taylor interface)
# amplifies roundoff; there s grows with it, and the bar with s.
def oracle_jitter_spread(p, phi, ux, uy, steps, base, seed=20150713):
    o = fast_oracle(p)
    o.init_phi(phi, ux, uy)
    o.step_jitter(steps, seed)
    f = o.fields()
    return {k: float(np.abs(f[k] - base[k]).max()) for k in base}


def bar64_long(k, o, spread, steps):
    rel_term = 1e-12 * max(steps / 100.0, 1.0) * float(np.abs(o[k]).max())
    if spread is not None and 10.0 * spread[k] > rel_term:
        return 10.0 * spread[k], "10s"
    return rel_term, "rel/100steps"


def check64_long(g, o, spread, tag, steps, keys=FIELDS):
    worst = []
    for k in keys:
        tol, term = bar64_long(k, o, spread, steps)
        err = float(np.abs(g[k] - o[k]).max())
        PARITY_LOG.append((tag, k, err, tol, term))
        print(f"PARITY64L {tag} {k} steps={steps} err={err:.3e} bar={tol:.3e} term={term} "
              f"ratio={err / tol if tol > 0 else float('inf'):.3f}")
        worst.append((err / tol if tol > 0 else float("inf"), k, err, tol, term))
    worst.sort(reverse=True)
    assert worst[0][0] <= 1.0, f"{tag}: {worst}"


def same_result(a, b, dtype, tag=""):
    """Two GPU runs of the same per-cell arithmetic in different kernels
    (single domain, batch, slabs): bit for bit in FP64, built without
    contracted multiply-adds, and in the 16-bit storage forms; within FP32
    rounding in FP32 (the FP32 parity bar, 1e-5 of the field's scale),
    where nvcc is free to contract a product and a sum into one FMA and
    does not do it the same way in every kernel."""
    a = np.asarray(a)
    b = np.asarray(b)
    if dtype == "f32":
        scale = max(1.0, float(np.abs(a).max()))
        err = float(np.abs(a.astype(np.float64) - b.astype(np.float64)).max())
        assert err <= 1e-5 * scale, (tag, err, scale)
    else:
        assert np.array_equal(a, b), tag


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
