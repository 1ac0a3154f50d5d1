"""The D3Q19 step on the GPU (lbm3_*) against the 3-D oracle (orc3.c),
element by element, and against what the model fixes in 3-D.

FP64 bar as in 2-D: max |gpu - oracle| <= max(1e-12 max |oracle|, 10 s),
s the oracle's own change under a 1-ulp perturbation of phi0.  FP32 within
1e-5 on phi and u.  A z-invariant 3-D run equals the 2-D GPU path; sum rho
and sum phi are conserved; a spherical droplet obeys dP = 2 sigma / R.
"""
import numpy as np
import pytest

import oracle
from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("phi", "rho", "p", "ux", "uy", "uz", "mu")


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm
    build.build()
    return lbm


def _p(**kw):
    d = dict(nx=12, ny=10, rho_A=1.0, rho_B=0.2, phi_A=1.0, phi_B=-1.0, sigma=0.01, W=3.0,
             M=0.1, tau_f=0.8, tau_g=0.9, gravity=0.0, rho_ref=0.6, bc_x=0, bc_y=0,
             u_wall_bottom=0.0, u_wall_top=0.0)
    d.update(kw)
    return d


def droplet3(nx, ny, nz, c, R, Wd, inside, outside):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx = np.minimum(np.abs(x - c[0]), nx - np.abs(x - c[0]))
    dy = np.minimum(np.abs(y - c[1]), ny - np.abs(y - c[1]))
    dz = np.minimum(np.abs(z - c[2]), nz - np.abs(z - c[2]))
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    return 0.5 * (inside + outside) + 0.5 * (inside - outside) * np.tanh(2.0 * (R - r) / Wd)


def _case(nx, ny, nz, seed, gravity=0.0):
    rng = np.random.default_rng(seed)
    p = _p(nx=nx, ny=ny, gravity=gravity)
    phi = droplet3(nx, ny, nz, (nx / 2 + 0.3, ny / 2 - 0.4, nz / 2 + 0.2), 0.3 * min(nx, ny, nz),
                   3.0, 1.0, -1.0)
    u = [0.01 * rng.standard_normal(phi.shape) for _ in range(3)]
    return p, phi, u


def _oracle(p, nz, phi, u, steps):
    o = oracle.Oracle3(p, nz)
    o.init_phi(phi, *u)
    o.step(steps)
    return o.fields()


def _spread(p, nz, phi, u, steps, base):
    rng = np.random.default_rng(5)
    pert = np.where(rng.uniform(size=phi.shape) < 0.5, np.nextafter(phi, np.inf),
                    np.nextafter(phi, -np.inf))
    f = _oracle(p, nz, pert, u, steps)
    return {k: float(np.abs(f[k] - base[k]).max()) for k in base}


def _gpu(L, p, nz, phi, u, steps, dtype):
    s = L.Sim3(p, nz, dtype)
    s.init_phi(phi, *u)
    s.step(steps)
    out = {k: v.double().cpu().numpy() for k, v in s.fields().items()}
    s.close()
    return out


# the last case: a deeper grid with odd sizes (33 planes)
CASES = [(12, 10, 9, 1, 0.0), (8, 6, 5, 2, 2e-5), (16, 8, 12, 3, -1e-5), (10, 9, 33, 4, 1e-5)]


@pytest.mark.parametrize("nx,ny,nz,seed,grav", CASES)
def test_3d_f64_matches_oracle(L, nx, ny, nz, seed, grav):
    p, phi, u = _case(nx, ny, nz, seed, grav)
    steps = 30
    ref = _oracle(p, nz, phi, u, steps)
    got = _gpu(L, p, nz, phi, u, steps, "f64")
    sp = _spread(p, nz, phi, u, steps, ref)
    for k in KEYS:
        tol = max(1e-12 * np.abs(ref[k]).max(), 10 * sp[k])
        err = np.abs(got[k] - ref[k]).max()
        assert err <= tol, (k, err, tol)


@pytest.mark.parametrize("nx,ny,nz,seed,grav", CASES[:2])
def test_3d_f32_matches_oracle(L, nx, ny, nz, seed, grav):
    p, phi, u = _case(nx, ny, nz, seed, grav)
    ref = _oracle(p, nz, phi, u, 30)
    got = _gpu(L, p, nz, phi, u, 30, "f32")
    for k in ("phi", "ux", "uy", "uz"):
        assert np.abs(got[k] - ref[k]).max() < 1e-5, k


def test_3d_z_invariant_equals_2d_path(L):
    p, phi, ux, uy = W.small_case(24, 16, seed=71)
    p = dict(p, bc_y=0)
    nz = 4
    a = L.Sim(p, "f64")
    a.init_phi(phi, ux, uy)
    a.step(50)
    r2 = {k: v.cpu().numpy() for k, v in a.fields().items()}
    rep = lambda x: np.repeat(x[None], nz, axis=0)
    r3 = _gpu(L, p, nz, rep(phi), [rep(ux), rep(uy), None], 50, "f64")
    for k in ("phi", "rho", "p", "ux", "uy", "mu"):
        scale = np.abs(r2[k]).max()
        assert np.abs(r3[k] - r2[k][None]).max() <= 1e-11 * scale, k
    assert np.abs(r3["uz"]).max() < 1e-15


def test_3d_conservation(L):
    p, phi, u = _case(16, 12, 10, 4, 1e-5)
    s = L.Sim3(p, 10, "f64")
    s.init_phi(phi, *u)
    m0, t0 = s.mass()
    s.step(500)
    m1, t1 = s.mass()
    assert abs(m1 - m0) <= 1e-12 * abs(m0)
    assert abs(t1 - t0) <= 1e-12 * np.abs(phi).sum()


def test_3d_laplace_law(L):
    """Spherical droplet of fluid A (phi = 1, rho = 1) in B (phi = 0, rho =
    0.2), R = 24, W = 3, sigma = 1e-3, lambda beta = 0.02, 96^3: the jump of
    the total pressure averaged over steps 3000-4000 is 2 sigma / R_eff."""
    n, R, sigma, Wd = 96, 24.0, 1e-3, 3.0
    beta = 12 * sigma / Wd
    p = _p(nx=n, ny=n, rho_B=0.2, phi_A=1.0, phi_B=0.0, sigma=sigma, W=Wd, M=0.02 / beta,
           tau_f=1.0, tau_g=1.0, rho_ref=1.0)
    s = L.Sim3(p, n, "f64")
    s.init_phi(droplet3(n, n, n, (n / 2, n / 2, n / 2), R, Wd, 1.0, 0.0))
    s.step(3000)
    vals = []
    for _ in range(5):
        dP, Re = s.laplace(n / 2, n / 2, n / 2, R)
        vals.append(dP * Re / (2 * sigma))
        s.step(250)
    ratio = float(np.mean(vals))
    print(f"3-D Laplace: dP R / (2 sigma) = {ratio:.4f}, R_eff = {Re:.3f}")
    assert abs(ratio - 1.0) < 0.03
    assert abs(Re - R) < 0.5


def test_3d_refusals(L):
    p = _p()
    with pytest.raises(L.LBMError):
        L.Sim3(dict(p, bc_y=1), 6, "f32")
    with pytest.raises(L.LBMError):
        L.Sim3(p, 6, "f16s")
    with pytest.raises(L.LBMError):
        L.Sim3(dict(p, gradp_lag=1), 6, "f32")
    with pytest.raises(L.LBMError):
        L.Sim3(p, 2, "f32")
