"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds no arithmetic of the scheme itself: only parameter sets
(plain dicts in the paper's notation) and initial order-parameter fields
(tanh-profiled droplets and layers, the initial conditions of Secs. 4.1-4.2).
Random draws use NumPy's PCG64 with explicit seeds.

Field layout: numpy arrays of shape [ny, nx], x fastest; node (i, j) sits at
x = i, y = j.
"""
from __future__ import annotations

import math

import numpy as np

PERIODIC = 0
WALL = 1


def _base(**kw) -> dict:
    d = dict(nx=64, ny=64, rho_A=1.0, rho_B=0.1, phi_A=1.0, phi_B=-1.0, sigma=0.01, W=4.0,
             M=0.1, tau_f=0.8, tau_g=0.8, gravity=0.0, rho_ref=1.0, bc_x=PERIODIC,
             bc_y=PERIODIC, u_wall_bottom=0.0, u_wall_top=0.0)
    d.update(kw)
    return d


# --------------------------------------------------------------- fields

def droplet_field(nx, ny, xc, yc, R, W, phi_A, phi_B, periodic=True):
    """phi = mean + (dphi/2) tanh(2 (R - r)/W) around (xc, yc), r measured to
    the nearest periodic image when periodic (initial condition of Sec. 4.2)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    dx = np.abs(x - xc)
    dy = np.abs(y - yc)
    if periodic:
        dx = np.minimum(dx, nx - dx)
        dy = np.minimum(dy, ny - dy)
    r = np.sqrt(dx * dx + dy * dy)
    return 0.5 * (phi_A + phi_B) + 0.5 * (phi_A - phi_B) * np.tanh(2.0 * (R - r) / W)


def layer_field(nx, ny, y_lo, y_hi, W, phi_A, phi_B):
    """Fluid A in y_lo <= y <= y_hi between two tanh interfaces (Sec. 4.1)."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    mid = 0.5 * (y_lo + y_hi)
    a = np.where(y <= mid, np.tanh(2.0 * (y - y_lo) / W), -np.tanh(2.0 * (y - y_hi) / W))
    return 0.5 * (phi_A + phi_B) + 0.5 * (phi_A - phi_B) * a


def multi_droplet_field(nx, ny, centres, radii, W, phi_A, phi_B):
    """phi = max over droplets of the tanh profile, background phi_B
    (periodic nearest-image distance).  Each droplet only touches a box of
    half-width R + 6W around its centre, where the profile differs from
    phi_B by more than 1e-10 relative."""
    mean, half = 0.5 * (phi_A + phi_B), 0.5 * (phi_A - phi_B)
    phi = np.full((ny, nx), float(phi_B))
    for (xc, yc), R in zip(centres, radii):
        h = int(math.ceil(R + 6 * W))
        xs = np.arange(int(math.floor(xc)) - h, int(math.floor(xc)) + h + 2)
        ys = np.arange(int(math.floor(yc)) - h, int(math.floor(yc)) + h + 2)
        dx = (xs - xc)[None, :]
        dy = (ys - yc)[:, None]
        r = np.sqrt(dx * dx + dy * dy)
        v = mean + half * np.tanh(2.0 * (R - r) / W)
        xi = np.mod(xs, nx)
        yi = np.mod(ys, ny)
        sub = phi[np.ix_(yi, xi)]
        phi[np.ix_(yi, xi)] = np.maximum(sub, v)
    return phi


def seeded_droplets(nx, ny, n, rmin, rmax, W, seed, max_tries=200000):
    """n non-overlapping droplets: centres uniform, radii uniform in
    [rmin, rmax], rejection-sampled so that centre distances (nearest
    periodic image) are at least R1 + R2 + 2W."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres, radii = [], []
    tries = 0
    while len(centres) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place droplets")
        R = rng.uniform(rmin, rmax)
        c = (rng.uniform(0, nx), rng.uniform(0, ny))
        ok = True
        for (x2, y2), R2 in zip(centres, radii):
            dx = abs(c[0] - x2)
            dy = abs(c[1] - y2)
            dx = min(dx, nx - dx)
            dy = min(dy, ny - dy)
            if dx * dx + dy * dy < (R + R2 + 2 * W) ** 2:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(R)
    return centres, radii


def rt_field(nx, ny, W, phi_A, phi_B, y0, amp):
    """Heavy fluid A above y_i(x) = y0 + amp cos(2 pi x / nx)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    yi = y0 + amp * np.cos(2.0 * np.pi * x / nx)
    return 0.5 * (phi_A + phi_B) + 0.5 * (phi_A - phi_B) * np.tanh(2.0 * (y - yi) / W)


# ------------------------------------------------------------ workloads

def droplet64():
    """Stationary droplet, 64x64 periodic, phi in [-1, 1], R = 16, W = 4,
    rho_A = 1, rho_B = 0.1, sigma = 0.01, M = 0.1, tau_f = tau_g = 0.8."""
    p = _base(nx=64, ny=64)
    phi = droplet_field(64, 64, 32.0, 32.0, 16.0, 4.0, 1.0, -1.0)
    return p, phi


def rayleigh_taylor(nx=256, ny=1024):
    """Rayleigh-Taylor, heavy over light, rho_A/rho_B = 3, W = 4,
    sigma = 5e-5, sqrt(g L) = 0.04, Re = 3000 with L = nx, periodic in x,
    no-slip walls at y = -1/2 and y = ny - 1/2.  g = 0.04^2/L,
    nu = 0.04 L / 3000 -> tau_f = 0.5 + 3 nu; tau_g = 0.8;
    M = 0.04 L / 1000; rho_ref = (rho_A + rho_B)/2."""
    L = float(nx)
    g = 0.04 ** 2 / L
    nu = 0.04 * L / 3000.0
    p = _base(nx=nx, ny=ny, rho_A=1.0, rho_B=1.0 / 3.0, sigma=5e-5, W=4.0,
              M=0.04 * L / 1000.0, tau_f=0.5 + 3.0 * nu, tau_g=0.8, gravity=g,
              rho_ref=0.5 * (1.0 + 1.0 / 3.0), bc_y=WALL)
    phi = rt_field(nx, ny, 4.0, 1.0, -1.0, ny / 2.0, 0.1 * nx)
    return p, phi


def precision(n=4096, n_drops=512, seed=1507035):
    """n x n periodic, n_drops droplets of radius U[8, 40] (fluid A inside),
    W = 4, rho_A = 1, rho_B = 0.01, sigma = 1e-3, M = 0.05, tau = 0.8."""
    p = _base(nx=n, ny=n, rho_A=1.0, rho_B=0.01, sigma=1e-3, M=0.05)
    centres, radii = seeded_droplets(n, n, n_drops, 8.0, 40.0, 4.0, seed)
    phi = multi_droplet_field(n, n, centres, radii, 4.0, 1.0, -1.0)
    return p, phi


def paper_droplet(R=25.0, n=100, Pe=50.0, Cn=4.0):
    """Stationary droplet of Sec. 4.2: 100x100 periodic, rho_A = 1,
    rho_B = 0.2, tau_f = tau_g = 1, phi_A = 1, phi_B = 0, sigma = 1e-3,
    W = Cn, lambda = 1/(Pe beta) with beta = 12 sigma / W (U_c = L_c = 1)."""
    sigma, W = 1e-3, float(Cn)
    beta = 12.0 * sigma / W
    p = _base(nx=n, ny=n, rho_A=1.0, rho_B=0.2, phi_A=1.0, phi_B=0.0, sigma=sigma, W=W,
              M=1.0 / (Pe * beta), tau_f=1.0, tau_g=1.0, rho_ref=1.0)
    phi = droplet_field(n, n, n / 2.0, n / 2.0, R, W, 1.0, 0.0)
    return p, phi


def paper_flat(nx=10, ny=100, Pe=50.0, Cn=4.0):
    """Flat interface of Sec. 4.1: fluid A in 25 <= y <= 75, periodic."""
    sigma, W = 1e-3, float(Cn)
    beta = 12.0 * sigma / W
    p = _base(nx=nx, ny=ny, rho_A=1.0, rho_B=0.2, phi_A=1.0, phi_B=0.0, sigma=sigma, W=W,
              M=1.0 / (Pe * beta), tau_f=1.0, tau_g=1.0, rho_ref=1.0)
    phi = layer_field(nx, ny, 25.0, 75.0, W, 1.0, 0.0)
    return p, phi


def droplet3_field(nx, ny, nz, centres, radii, W, phi_A, phi_B):
    """phi of spherical droplets (maximum over droplets of the tanh profile,
    nearest periodic image), background phi_B; array [nz, ny, nx].  Each
    droplet is evaluated on its periodic bounding box of radius R + 10W;
    beyond it tanh(2(R - r)/W) rounds to -1 in double precision, so the
    field equals the direct evaluation."""
    mid, half = 0.5 * (phi_A + phi_B), 0.5 * (phi_A - phi_B)
    out = np.full((nz, ny, nx), float(phi_B))
    for (cx, cy, cz), R in zip(centres, radii):
        reach = R + 10.0 * W
        axes = []
        for c, n in ((cz, nz), (cy, ny), (cx, nx)):
            lo, hi = int(np.floor(c - reach)), int(np.ceil(c + reach))
            idx = np.arange(lo, hi + 1) if hi - lo + 1 < n else np.arange(n)
            d = np.abs(idx.astype(np.float64) - c)
            if hi - lo + 1 >= n:
                d = np.minimum(d, n - d)
            axes.append((np.mod(idx, n), d))
        (iz, dz), (iy, dy), (ix, dx) = axes
        r = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        box = mid + half * np.tanh(2.0 * (R - r) / W)
        sub = out[np.ix_(iz, iy, ix)]
        out[np.ix_(iz, iy, ix)] = np.maximum(sub, box)
    return out


def precision3d(n=256, n_drops=64, seed=1507037):
    """The precision workload's 3-D analogue: n^3 periodic, n_drops spherical
    droplets of fluid A (phi = 1), radii U[6, 16], centres uniform and
    rejection-sampled at least R1 + R2 + 2W apart (PCG64 seed), background
    phi = -1; W = 4, rho_A = 1, rho_B = 0.01, sigma = 1e-3, M = 0.05,
    tau = 0.8.  Returns (params, phi [nz, ny, nx], nz)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Wd = 4.0
    centres, radii = [], []
    tries = 0
    while len(centres) < n_drops and tries < 200000:
        tries += 1
        R = rng.uniform(6.0, 16.0)
        c = rng.uniform(0, n, size=3)
        ok = True
        for c2, R2 in zip(centres, radii):
            d = np.abs(c - c2)
            d = np.minimum(d, n - d)
            if np.sqrt((d * d).sum()) < R + R2 + 2 * Wd:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(R)
    p = _base(nx=n, ny=n, rho_A=1.0, rho_B=0.01, sigma=1e-3, M=0.05)
    return p, droplet3_field(n, n, n, centres, radii, Wd, 1.0, -1.0), n


def paper_bubble(nx=160, ny=480, R=32.0, yc=120.0, Pe=50.0, Cn=4.0):
    """Bubble rising under buoyancy, Sec. 4.3: 160 x 480 periodic, a light
    bubble of fluid B (phi_B = 0, rho_B = 0.5) of radius 32 in fluid A
    (phi_A = 1, rho_A = 1); F_b,y = -(rho - rho_A) g with g = 1e-5;
    tau_f = tau_g = 1, sigma = 1e-3, Pe = 50, Cn = 4 (lambda = 1/(Pe beta)).
    The paper does not give the bubble's starting point: it is centred in
    x (x = nx/2, which keeps the lattice mirror x -> nx - x exact) at
    y = 120, a quarter of the way up."""
    sigma, W = 1e-3, float(Cn)
    beta = 12.0 * sigma / W
    p = _base(nx=nx, ny=ny, rho_A=1.0, rho_B=0.5, phi_A=1.0, phi_B=0.0, sigma=sigma, W=W,
              M=1.0 / (Pe * beta), tau_f=1.0, tau_g=1.0, gravity=1e-5, rho_ref=1.0)
    phi = droplet_field(nx, ny, nx / 2.0, yc, R, W, 0.0, 1.0)
    return p, phi


def paper_phase_separation(gamma=1.0, Pe=50.0, Cn=4.0, eps=0.1, n=100):
    """Phase separation, Sec. 4.4: n x n periodic (100 in the paper),
    phi = 0.5 [1 + eps sin(4 pi x/Lx) cos(4 pi y/Ly)] with eps = 0.1;
    rho_A = 1, phi_A = 1, phi_B = 0, tau_f = tau_g = 1, sigma = 1e-3;
    lambda beta = 1/Pe (0.02 and 0.005), W = Cn (4 and 8), rho_r = 2 and 5,
    i.e. gamma = rho_r - 1 = 1 and 4 (Eq. 17 with phi_B = 0)."""
    sigma, W = 1e-3, float(Cn)
    beta = 12.0 * sigma / W
    p = _base(nx=n, ny=n, rho_A=1.0, rho_B=1.0 / (1.0 + gamma), phi_A=1.0, phi_B=0.0,
              sigma=sigma, W=W, M=1.0 / (Pe * beta), tau_f=1.0, tau_g=1.0, rho_ref=1.0)
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x)
    phi = 0.5 * (1.0 + eps * np.sin(4 * np.pi * X / n) * np.cos(4 * np.pi * Y / n))
    return p, phi


def small_case(nx, ny, seed, walls=False, gravity=0.0, u_wall=0.0, rho_ratio=10.0):
    """A small seeded domain for parity: an off-centre droplet with a
    seeded velocity perturbation, phi in [-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = 0.3 * min(nx, ny)
    xc = nx / 2.0 + rng.uniform(-1, 1)
    yc = ny / 2.0 + rng.uniform(-1, 1)
    p = _base(nx=nx, ny=ny, rho_A=1.0, rho_B=1.0 / rho_ratio, sigma=0.01, W=4.0, M=0.1,
              tau_f=0.8, tau_g=0.9, gravity=gravity, rho_ref=0.5 * (1.0 + 1.0 / rho_ratio),
              bc_y=WALL if walls else PERIODIC, u_wall_bottom=-u_wall, u_wall_top=u_wall)
    phi = droplet_field(nx, ny, xc, yc, R, 4.0, 1.0, -1.0, periodic=not walls)
    ux = 0.01 * rng.standard_normal((ny, nx))
    uy = 0.01 * rng.standard_normal((ny, nx))
    return p, phi, ux, uy


def batch_domains(n=1024, seed=1507036, sides=tuple(range(64, 513, 32)), max_side=None):
    """n independent periodic domains: nx, ny uniform over `sides`; half
    hold a centred tanh droplet of radius U[0.2, 0.35] x min side, half a
    flat layer of fluid A in ny/4 <= y < 3ny/4 (Sec. 4.1 shape); rho_A = 1,
    rho_A/rho_B log-uniform in [1, 100]; sigma U[1e-4, 1e-2]; M U[0.01, 0.2];
    tau = 0.8; phi in [-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = [s for s in sides if max_side is None or s <= max_side]
    out = []
    for _ in range(n):
        nx = int(rng.choice(sides))
        ny = int(rng.choice(sides))
        ratio = float(np.exp(rng.uniform(0.0, np.log(100.0))))
        sigma = float(rng.uniform(1e-4, 1e-2))
        M = float(rng.uniform(0.01, 0.2))
        p = _base(nx=nx, ny=ny, rho_A=1.0, rho_B=1.0 / ratio, sigma=sigma, W=4.0, M=M,
                  tau_f=0.8, tau_g=0.8)
        if rng.uniform() < 0.5:
            R = float(rng.uniform(0.2, 0.35)) * min(nx, ny)
            phi = droplet_field(nx, ny, nx / 2.0, ny / 2.0, R, 4.0, 1.0, -1.0)
        else:
            phi = layer_field(nx, ny, ny / 4.0, 3.0 * ny / 4.0 - 1.0, 4.0, 1.0, -1.0)
        out.append((p, phi))
    return out


def shear_droplet(n=512, R=64.0, u_wall=0.01, rho_ratio=10.0):
    """Droplet in shear: n x n, centred droplet of radius R (W = 4), walls at
    y = -1/2 and n - 1/2 moving at -u_wall (bottom) and +u_wall (top),
    rho_A/rho_B = rho_ratio, sigma = 1e-3, M = 0.05, tau_f = tau_g = 0.8,
    periodic in x."""
    p = _base(nx=n, ny=n, rho_A=1.0, rho_B=1.0 / rho_ratio, sigma=1e-3, W=4.0, M=0.05,
              tau_f=0.8, tau_g=0.8, bc_y=WALL, u_wall_bottom=-u_wall, u_wall_top=u_wall,
              rho_ref=1.0)
    phi = droplet_field(n, n, n / 2.0, n / 2.0, R, 4.0, 1.0, -1.0, periodic=False)
    return p, phi
