"""Paper experiments reproduced on the GPU path (FP64).

Table I (Sec. 4.2): stationary droplet, 100 x 100, R = 25, rho_A = 1,
rho_B = 0.2, tau = 1, phi_A = 1, phi_B = 0, sigma = 1e-3, lambda = 1/(Pe beta).
The paper reports sigma_LBM = R dP = 0.992e-3 (Pe = 50, 125, 200 at Cn = 4)
and 0.993e-3, 0.989e-3 (Cn = 6, 8 at Pe = 200).  dP is the jump of the total
pressure of Sec. 4.2, averaged over steps 16000-20000 (the start from p = 0
leaves slowly damped acoustic oscillations).

Sec. 4.1: the flat interface keeps the tanh profile of Eq. 6 (Cn = 4, 8).

Sec. 4.3 (bubble rising, 160 x 480) and Sec. 4.4 (phase separation,
100 x 100, gamma = 1 and 4): the GPU path against the oracle element by
element early in the run, and over the paper's time spans against what
the model fixes (linear growth rate with the (1 + gamma phi) factor of
Eq. 19, conservation, the buoyancy impulse, mirror symmetry, separation
earlier at the larger gamma, relaxation to rest).
"""
import math

import numpy as np
import pytest

from helpers import check64_long, fast_oracle, linear_rate, mode_amplitude, oracle_jitter_spread
from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (Pe, Cn, paper's sigma_LBM / sigma, droplet radius), the paper's values
# from tests/golden/table1_surface_tension.json.  The paper's radii range
# from 20 to 40 without saying which Table I used; R = 40 keeps the
# interface width W = Cn below 0.2 R for Cn = 6 and 8.
def _table1():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "table1_surface_tension.json")) as f:
        g = json.load(f)
    return [(c["Pe"], c["Cn"], c["sigma_lbm_over_1e-3"], 25.0 if c["Cn"] == 4.0 else 40.0)
            for c in g["cases"]]


TABLE1 = _table1()


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm
    build.build()
    return lbm


@pytest.mark.parametrize("Pe,Cn,paper,R", TABLE1)
def test_table1_laplace_law(L, Pe, Cn, paper, R):
    p, phi = W.paper_droplet(R=R, Pe=Pe, Cn=Cn)
    s = L.Sim(p, "f64")
    s.init_phi(phi)
    s.step(16000)
    vals = []
    for _ in range(9):
        dP, Re = s.laplace(50.0, 50.0, R)
        vals.append(dP * Re / 1e-3)
        s.step(500)
    ratio = float(np.mean(vals))
    print(f"Pe={Pe} Cn={Cn} R={R}: sigma_LBM/sigma = {ratio:.4f} (paper {paper})")
    assert abs(ratio - 1.0) < 0.015
    assert abs(ratio - paper) < 0.02


@pytest.mark.parametrize("Cn,Pe,tol", [(4.0, 50.0, 1e-2), (8.0, 1000.0, 2.5e-3)])
def test_flat_interface_profile_gpu(L, Cn, Pe, tol):
    p, phi = W.paper_flat(Cn=Cn, Pe=Pe)
    s = L.Sim(p, "f64")
    s.init_phi(phi)
    s.step(3000)
    ph = s.fields(("phi",))["phi"].cpu().numpy()
    y = np.arange(100, dtype=float)
    prof = np.where(y <= 50, 0.5 + 0.5 * np.tanh(2 * (y - 25) / Cn), 0.5 - 0.5 * np.tanh(2 * (y - 75) / Cn))
    assert np.abs(ph - prof[:, None]).max() < tol


def _mode(n):
    x = np.arange(n)
    X, Y = np.meshgrid(x, x)
    return np.sin(4 * np.pi * X / n) * np.cos(4 * np.pi * Y / n)


@pytest.mark.parametrize("dtype,tol", [("f64", 0.01), ("f32", 0.03)])
@pytest.mark.parametrize("gamma", [1.0, 4.0])
def test_phase_separation_linear_growth_gpu(L, gamma, dtype, tol):
    p, phi = W.paper_phase_separation(gamma=gamma, eps=2e-4)
    n = p["nx"]
    mode = _mode(n)
    s = L.Sim(p, dtype)
    s.init_phi(phi)
    amps = []
    for t in (300, 1300):
        s.step(t - s.step_count)
        amps.append(mode_amplitude(s.fields(("phi",))["phi"].double().cpu().numpy(), mode))
    rate = math.log(amps[1] / amps[0]) / 1000.0
    a = 4 * np.pi / n
    assert rate == pytest.approx(linear_rate(p, 0.5, a, a), rel=tol)


def test_phase_separation_paper_case(L):
    """Sec. 4.4 at Pe = 50, Cn = 4, eps = 0.1: the GPU matches the oracle
    through the fast transient (2500 steps, the long-run FP64 bar: the
    decomposition amplifies roundoff); over 20000 steps both gamma
    separate, gamma = 4 first, sum phi stays put and the flow comes to rest."""
    first = {}
    for gamma in (1.0, 4.0):
        p, phi = W.paper_phase_separation(gamma=gamma)
        s = L.Sim(p, "f64")
        s.init_phi(phi)
        s.step(2500)
        g = {k: v.cpu().numpy() for k, v in s.fields().items()}
        o = fast_oracle(p)
        o.init_phi(phi)
        o.step(2500)
        ref = o.fields()
        check64_long(g, ref, oracle_jitter_spread(p, phi, None, None, 2500, ref),
                     f"phase separation gamma={gamma}", 2500)
        s2 = L.Sim(p, "f64")
        s2.init_phi(phi)
        m0, t0 = s2.mass()
        first[gamma] = None
        while s2.step_count < 20000:
            s2.step(250)
            ph = s2.fields(("phi",))["phi"].cpu().numpy()
            if first[gamma] is None and ph.max() - ph.min() > 0.9:
                first[gamma] = s2.step_count
        m1, t1 = s2.mass()
        fl = s2.fields(("phi", "ux", "uy"))
        assert abs(t1 - t0) <= 1e-12 * t0 and abs(m1 - m0) <= 1e-12 * m0
        assert float(fl["phi"].max()) > 0.95 and float(fl["phi"].min()) < 0.05
        assert float(max(fl["ux"].abs().max(), fl["uy"].abs().max())) < 1e-6
        assert first[gamma] is not None
    assert first[4.0] < first[1.0]


def test_bubble_rising(L):
    """Sec. 4.3: FP64 GPU against the oracle for 300 steps (the long-run FP64
    bar), then to the
    paper's first snapshot (t = 10^4): conservation, the buoyancy impulse in
    the total momentum, mirror symmetry about x = nx/2, the bubble rising
    relative to the mean flow.  FP32 against FP64 at t = 10^4: the largest
    phi difference sits on the moving interface, where d phi/dy is about
    1/(2W) = 0.125 per cell; the bound 5e-3 is an interface offset of 0.04
    cells (measured: 1.0e-3, i.e. 0.008 cells)."""
    p, phi = W.paper_bubble()
    ny, nx = phi.shape
    s = L.Sim(p, "f64")
    s.init_phi(phi)
    fl0 = {k: v.cpu().numpy() for k, v in s.fields().items()}
    mom0 = float(np.sum(fl0["rho"] * fl0["uy"]))
    m0, t0 = s.mass()
    s.step(300)
    g = {k: v.cpu().numpy() for k, v in s.fields().items()}
    o = fast_oracle(p)
    o.init_phi(phi)
    o.step(300)
    ref = o.fields()
    check64_long(g, ref, oracle_jitter_spread(p, phi, None, None, 300, ref), "bubble, 300 steps",
                 300)
    T = 10000
    s.step(T - 300)
    fl = {k: v.cpu().numpy() for k, v in s.fields().items()}
    m1, t1 = s.mass()
    assert abs(m1 - m0) <= 1e-12 * m0 and abs(t1 - t0) <= 1e-12 * t0
    impulse = T * p["gravity"] * (p["rho_A"] - p["rho_B"]) * np.sum(1.0 - phi)
    gain = float(np.sum(fl["rho"] * fl["uy"])) - mom0
    assert gain == pytest.approx(impulse, rel=5e-3)
    mirror = (-np.arange(nx)) % nx
    assert np.abs(fl["phi"] - fl["phi"][:, mirror]).max() < 1e-11
    b = 1.0 - fl["phi"]
    y = np.arange(ny)[:, None]
    b0 = 1.0 - phi
    assert np.sum(b * y) / np.sum(b) > np.sum(b0 * y) / np.sum(b0) + 1.0
    assert np.sum(b * fl["uy"]) / np.sum(b) > np.mean(fl["uy"])
    s32 = L.Sim(p, "f32")
    s32.init_phi(phi)
    s32.step(T)
    ph32 = s32.fields(("phi",))["phi"].double().cpu().numpy()
    assert np.abs(ph32 - fl["phi"]).max() < 5e-3
