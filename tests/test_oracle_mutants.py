"""Mutation test of the oracle's pins.

Each mutant is the oracle built with one plausible mistake planted
(``-DORC_MUTANT=k`` in ``oracle/orc.c``): a dropped term, a flipped sign, a
swapped velocity component, a wrong constant.  The test runs a quick battery
of the same pins the oracle tests use and requires that each mutant fails at
least one, while the unmutated oracle passes all of them.  Nothing here runs
on a GPU.
"""
import math
import os

import numpy as np
import pytest

from paper_1507_03521_gb300 import workloads as W

CS2 = 1.0 / 3.0
MUTANTS = {
    1: "Gamma_i = 1 (s_i dropped)",
    2: "sign of the grad rho term of F_i",
    3: "half force missing from u (Eq. 31)",
    4: "(1 - 1/2tau) forcing prefactor dropped",
    5: "H_0 uses w_0 instead of 1 - w_0",
    6: "gradient components swapped",
    7: "sign of the gamma term of F_i",
    8: "lap mu term missing from p (Eq. 32)",
    9: "1/rho missing from G_i",
    10: "moving-wall term missing from bounce-back",
    11: "sign of the kappa lap phi term of mu",
    12: "kappa off by a factor 2",
}


def _base(**kw):
    d = dict(nx=16, ny=12, rho_A=1.0, rho_B=0.1, phi_A=1.0, phi_B=-1.0, sigma=0.01, W=4.0,
             M=0.1, tau_f=0.8, tau_g=0.8, gravity=0.0, rho_ref=1.0, bc_x=0, bc_y=0,
             u_wall_bottom=0.0, u_wall_top=0.0)
    d.update(kw)
    return d


def pin_identities(orc, lib):
    cx, cy, w = orc.lattice()
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = dict(alpha=rng.uniform(0.2, 3), gamma=rng.uniform(0.5, 5), lam=rng.uniform(0.01, 1),
                 phi=rng.uniform(-1, 1), mu=rng.normal() * 1e-2, p=rng.normal() * 1e-3,
                 rho=rng.uniform(0.05, 1.5), ux=rng.uniform(-.1, .1), uy=rng.uniform(-.1, .1),
                 Fx=rng.normal() * 1e-3, Fy=rng.normal() * 1e-3, grhx=rng.normal() * .1,
                 grhy=rng.normal() * .1, lmu=rng.normal() * 1e-3, gpx=rng.normal() * 1e-3,
                 gpy=rng.normal() * 1e-3)
        args = [a[k] for k in ("alpha", "gamma", "lam", "phi", "mu", "p", "rho", "ux", "uy", "Fx",
                               "Fy", "grhx", "grhy", "lmu", "gpx", "gpy")]
        feq, geq, Fi, Gi = orc.cell_terms(*args, lib=lib)
        args0 = list(args)
        args0[13] = 0.0
        _, _, F0, _ = orc.cell_terms(*args0, lib=lib)
        F1 = Fi - F0
        checks = [
            abs(geq.sum() - a["phi"]) < 1e-15,
            abs(F0.sum() - CS2 * (a["ux"] * a["grhx"] + a["uy"] * a["grhy"])) < 1e-15,
            abs((cx * F0).sum() - CS2 * a["Fx"]) < 1e-15,
            abs(F1.sum() + CS2 * a["rho"] * a["gamma"] * a["lam"] * a["lmu"]) < 1e-17,
            abs((cx * Gi).sum() - a["phi"] / a["rho"] * (a["Fx"] - a["gpx"])) < 1e-15,
        ]
        if not all(checks):
            return False
    return True


def pin_stencil_symbol(orc, lib):
    nx, ny = 24, 20
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    a, b = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    c = np.cos(a * x + b * y + 0.3)
    s = np.sin(a * x + b * y + 0.3)
    gx, gy, lap = orc.stencils(c, lib=lib)
    gxs = 3.0 * np.sin(a) * (2 / 9 + np.cos(b) / 9)
    gys = 3.0 * np.sin(b) * (2 / 9 + np.cos(a) / 9)
    return np.allclose(gx, -gxs * s, atol=1e-13) and np.allclose(gy, -gys * s, atol=1e-13)


def pin_body_force(orc, lib):
    g = 2e-5
    o = orc.Oracle(_base(gravity=g, rho_ref=0.2, tau_f=0.7), lib=lib)
    o.init_phi(np.full((12, 16), 0.5))
    rho = 0.1 + 1.5 * 0.45
    o.step(10)
    return np.allclose(o.fields()["uy"], 10.5 * (-(rho - 0.2) * g) / rho, rtol=1e-11, atol=0)


def pin_couette(orc, lib):
    U, ny = 0.01, 12
    o = orc.Oracle(_base(nx=5, ny=ny, bc_y=1, u_wall_bottom=-U, u_wall_top=U), lib=lib)
    o.init_phi(np.full((ny, 5), 0.3))
    o.step(8000)
    y = np.arange(ny, dtype=float)
    return np.allclose(o.fields()["ux"][:, 0], -U + 2 * U * (y + 0.5) / ny, rtol=0, atol=1e-15)


def pin_profile(orc, lib):
    p, phi = W.paper_flat()
    o = orc.Oracle(p, lib=lib)
    o.init_phi(phi)
    o.step(3000)
    ph = o.fields()["phi"]
    y = np.arange(100, dtype=float)
    prof = np.where(y <= 50, 0.5 + 0.5 * np.tanh((y - 25) / 2), 0.5 - 0.5 * np.tanh((y - 75) / 2))
    return bool(np.isfinite(ph).all() and np.abs(ph - prof[:, None]).max() < 1e-2)


def pin_decay(orc, lib):
    nx = 32
    p = dict(nx=nx, ny=5, rho_A=1.0, rho_B=0.2, phi_A=1.0, phi_B=0.0, sigma=1e-3, W=4.0, M=0.2,
             tau_f=1.0, tau_g=1.0, gravity=0.0, rho_ref=1.0, bc_x=0, bc_y=0,
             u_wall_bottom=0.0, u_wall_top=0.0)
    o = orc.Oracle(p, lib=lib)
    x = np.arange(nx)
    o.init_phi(np.tile(1.0 + 1e-4 * np.cos(2 * np.pi * x / nx), (5, 1)))
    amps = []
    for t in (400, 2400):
        o.step(t - o.step_count)
        ph = o.fields()["phi"][2]
        amps.append(2.0 / nx * np.sum((ph - ph.mean()) * np.cos(2 * np.pi * x / nx)))
    if not (amps[0] > 0 and amps[1] > 0):
        return False
    rate = math.log(amps[0] / amps[1]) / 2000
    beta, kappa = 12e-3 / 4.0, 1.5e-3 * 4.0
    s2 = 4 * math.sin(math.pi / nx) ** 2
    return abs(rate / (5 * 0.2 * s2 * (2 * beta + kappa * s2)) - 1) < 0.03


PINS = [pin_identities, pin_stencil_symbol, pin_body_force, pin_couette, pin_profile, pin_decay]


def test_unmutated_oracle_passes_battery(orc):
    for pin in PINS:
        assert pin(orc, None), pin.__name__


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_mutant_is_caught(orc, k, tmp_path):
    lib = orc.build_mutant(k, str(tmp_path))
    failed = []
    for pin in PINS:
        try:
            ok = pin(orc, lib)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
            break
    assert failed, f"mutant {k} ({MUTANTS[k]}) passed every pin"
