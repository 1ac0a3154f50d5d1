"""Pins of the oracle's per-cell formulas against the exact discrete moment
identities the paper prints in its appendix.

- Eqs. 49-51: moments of f^eq (Eq. 24).
- Eqs. 52-54: moments of the source F_i (Eq. 28), split into F^(0) and F^(1)
  as in Eq. 43.
- Eq. 72: moments of g^eq (Eqs. 25-27); Eq. 73: moments of G_i (Eq. 29).

These hold exactly (to roundoff) for the zeroth and first moments only with
Gamma_i = 1 + s_i(u), which is how the oracle reads the undefined Gamma_i;
the second moment of F^(0) (Eq. 54) holds to O(u^3), the order the
Chapman-Enskog analysis keeps.  A dropped term, a wrong sign or a swapped
velocity component in any of Eqs. 24-29 breaks at least one identity.
"""
import math

import numpy as np
import pytest

CS2 = 1.0 / 3.0


def _lattice_from_paper():
    # End of Sec. 3: c_0 = 0; c_i = (cos, sin)[(i-1) pi/2] for i = 1..4;
    # c_i = sqrt(2) (cos, sin)[(2i-1) pi/4] for i = 5..8.
    cx, cy = [0], [0]
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        cx.append(round(math.cos(a)))
        cy.append(round(math.sin(a)))
    for i in range(5, 9):
        a = (2 * i - 1) * math.pi / 4
        cx.append(round(math.sqrt(2) * math.cos(a)))
        cy.append(round(math.sqrt(2) * math.sin(a)))
    w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    return np.array(cx), np.array(cy), np.array(w)


def test_lattice_tables(orc):
    cx, cy, w = orc.lattice()
    pcx, pcy, pw = _lattice_from_paper()
    assert list(cx) == list(pcx) and list(cy) == list(pcy)
    assert np.allclose(w, pw, rtol=0, atol=1e-17)
    # isotropy up to fourth order (what D2Q9 with c_s^2 = 1/3 must satisfy)
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * cx).sum()) < 1e-16 and abs((w * cy).sum()) < 1e-16
    assert abs((w * cx * cx).sum() - CS2) < 1e-15
    assert abs((w * cx * cy).sum()) < 1e-16
    assert abs((w * cx ** 4).sum() - 3 * CS2 ** 2) < 1e-15
    assert abs((w * cx ** 2 * cy ** 2).sum() - CS2 ** 2) < 1e-15


def _random_state(rng, umax=0.1):
    return dict(alpha=rng.uniform(0.2, 3), gamma=rng.uniform(-1, 5), lam=rng.uniform(0.01, 1),
                phi=rng.uniform(-1, 1), mu=rng.normal() * 1e-2, p=rng.normal() * 1e-3,
                rho=rng.uniform(0.05, 1.5), ux=rng.uniform(-umax, umax), uy=rng.uniform(-umax, umax),
                Fx=rng.normal() * 1e-3, Fy=rng.normal() * 1e-3, grhx=rng.normal() * 0.1,
                grhy=rng.normal() * 0.1, lmu=rng.normal() * 1e-3, gpx=rng.normal() * 1e-3,
                gpy=rng.normal() * 1e-3)


def _terms(orc, s, **over):
    d = dict(s)
    d.update(over)
    return orc.cell_terms(d["alpha"], d["gamma"], d["lam"], d["phi"], d["mu"], d["p"], d["rho"],
                          d["ux"], d["uy"], d["Fx"], d["Fy"], d["grhx"], d["grhy"], d["lmu"],
                          d["gpx"], d["gpy"])


@pytest.mark.parametrize("seed", range(20))
def test_feq_geq_moments(orc, seed):
    rng = np.random.default_rng(seed)
    cx, cy, w = orc.lattice()
    s = _random_state(rng)
    feq, geq, _, _ = _terms(orc, s)
    rho, p, ux, uy, phi, mu, al = s["rho"], s["p"], s["ux"], s["uy"], s["phi"], s["mu"], s["alpha"]
    tol = 1e-15
    # Eq. 49
    assert abs(feq.sum() - p) < tol
    assert abs((cx * feq).sum() - CS2 * rho * ux) < tol
    assert abs((cy * feq).sum() - CS2 * rho * uy) < tol
    # Eq. 50
    assert abs((cx * cx * feq).sum() - (CS2 * p + CS2 * rho * ux * ux)) < tol
    assert abs((cy * cy * feq).sum() - (CS2 * p + CS2 * rho * uy * uy)) < tol
    assert abs((cx * cy * feq).sum() - CS2 * rho * ux * uy) < tol
    # Eq. 51 (off-diagonal third moments, which D2Q9 reproduces)
    assert abs((cx * cx * cy * feq).sum() - CS2 ** 2 * rho * uy) < tol
    assert abs((cx * cy * cy * feq).sum() - CS2 ** 2 * rho * ux) < tol
    # Eq. 72
    assert abs(geq.sum() - phi) < tol
    assert abs((cx * geq).sum() - phi * ux) < tol
    assert abs((cy * geq).sum() - phi * uy) < tol
    assert abs((cx * cx * geq).sum() - (phi * ux * ux + CS2 * al * mu)) < tol
    assert abs((cy * cy * geq).sum() - (phi * uy * uy + CS2 * al * mu)) < tol
    assert abs((cx * cy * geq).sum() - phi * ux * uy) < tol


@pytest.mark.parametrize("seed", range(20))
def test_source_moments(orc, seed):
    rng = np.random.default_rng(100 + seed)
    cx, cy, w = orc.lattice()
    s = _random_state(rng)
    rho, ux, uy, Fx, Fy = s["rho"], s["ux"], s["uy"], s["Fx"], s["Fy"]
    grx, gry, lmu, gam, lam = s["grhx"], s["grhy"], s["lmu"], s["gamma"], s["lam"]
    _, _, F0, G = _terms(orc, s, lmu=0.0)       # F^(0): the lmu term removed
    _, _, Fall, _ = _terms(orc, s)
    F1 = Fall - F0                                # F^(1) of Eq. 43
    udr = ux * grx + uy * gry
    scale = 1e-3
    tol = 1e-15 * max(1.0, scale)
    # Eq. 52
    assert abs(F0.sum() - CS2 * udr) < tol
    assert abs(F1.sum() - (-CS2 * rho * gam * lam * lmu)) < 1e-17
    # Eq. 53
    assert abs((cx * F0).sum() - CS2 * Fx) < tol
    assert abs((cy * F0).sum() - CS2 * Fy) < tol
    assert abs((cx * F1).sum()) < 1e-18 and abs((cy * F1).sum()) < 1e-18
    # Eq. 54, second moment of F^(1), exact
    assert abs((cx * cx * F1).sum() - (-CS2 ** 2 * rho * gam * lam * lmu)) < 1e-18
    assert abs((cx * cy * F1).sum()) < 1e-18
    # Eq. 73
    phi, gpx, gpy = s["phi"], s["gpx"], s["gpy"]
    assert abs(G.sum()) < 1e-17
    assert abs((cx * G).sum() - phi / rho * (Fx - gpx)) < 1e-15
    assert abs((cy * G).sum() - phi / rho * (Fy - gpy)) < 1e-15


def test_source_second_moment_order_u3(orc):
    """Eq. 54 for F^(0): the residual is O(u^3).  Halving u divides it by 8."""
    cx, cy, w = orc.lattice()
    rng = np.random.default_rng(7)
    s = _random_state(rng)
    res = []
    for scale in (1.0, 0.5, 0.25):
        d = dict(s, ux=0.08 * scale, uy=-0.05 * scale, lmu=0.0)
        _, _, F0, _ = _terms(orc, d)
        Fpx = d["Fx"] + CS2 * d["grhx"]
        Fpy = d["Fy"] + CS2 * d["grhy"]
        udr = d["ux"] * d["grhx"] + d["uy"] * d["grhy"]
        exx = CS2 * 2 * Fpx * d["ux"] + CS2 ** 2 * udr
        exy = CS2 * (Fpx * d["uy"] + Fpy * d["ux"])
        res.append((abs((cx * cx * F0).sum() - exx), abs((cx * cy * F0).sum() - exy)))
    for k in range(2):
        assert res[0][k] / res[1][k] == pytest.approx(8.0, rel=1e-6)
        assert res[1][k] / res[2][k] == pytest.approx(8.0, rel=1e-6)


def test_gamma_reading_is_forced(orc):
    """With u = 0 the first moment of F^(0) is c_s^2 F for any Gamma_i with
    Gamma_i(0) = 1; at u != 0 the identity only holds with the s_i(u) term.
    Check that the oracle's F_i differs from the truncated reading
    Gamma_i = 1 + c_i.u/c_s^2 by exactly the quadratic part of s_i."""
    cx, cy, w = orc.lattice()
    s = _random_state(np.random.default_rng(3))
    s.update(lmu=0.0, grhx=0.0, grhy=0.0)
    _, _, F0, _ = _terms(orc, s)
    ux, uy = s["ux"], s["uy"]
    cu = cx * ux + cy * uy
    quad = (cu * cu - CS2 * (ux * ux + uy * uy)) / (2 * CS2 ** 2)
    trunc = ((cx - ux) * s["Fx"] + (cy - uy) * s["Fy"]) * w * (1 + cu / CS2)
    np.testing.assert_allclose(F0 - trunc, ((cx - ux) * s["Fx"] + (cy - uy) * s["Fy"]) * w * quad,
                               rtol=0, atol=1e-18)
