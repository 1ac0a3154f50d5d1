"""Paper experiments reproduced on the GPU path (FP64).

Table I (Sec. 4.2): stationary droplet, 100 x 100, R = 25, rho_A = 1,
rho_B = 0.2, tau = 1, phi_A = 1, phi_B = 0, sigma = 1e-3, lambda = 1/(Pe beta).
The paper reports sigma_LBM = R dP = 0.992e-3 (Pe = 50, 125, 200 at Cn = 4)
and 0.993e-3, 0.989e-3 (Cn = 6, 8 at Pe = 200).  dP is the jump of the total
pressure of Sec. 4.2, averaged over steps 16000-20000 (the start from p = 0
leaves slowly damped acoustic oscillations).

Sec. 4.1: the flat interface keeps the tanh profile of Eq. 6 (Cn = 4, 8).
"""
import numpy as np
import pytest

from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (Pe, Cn, paper's sigma_LBM / sigma, droplet radius).  The paper's radii
# range from 20 to 40 without saying which Table I used; R = 40 keeps the
# interface width W = Cn below 0.2 R for Cn = 6 and 8.
TABLE1 = [(50.0, 4.0, 0.992, 25.0), (125.0, 4.0, 0.992, 25.0), (200.0, 4.0, 0.992, 25.0),
          (200.0, 6.0, 0.993, 40.0), (200.0, 8.0, 0.989, 40.0)]


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
