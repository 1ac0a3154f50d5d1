"""Plain PyTorch (CPU, FP64) statement of one time step, differentiable.

TEST INFRASTRUCTURE ONLY, like the C oracle: it exists so that autograd can
provide the reference vector-Jacobian products the hand-written adjoint of
the CUDA library is checked against.  It is the same scheme as ``orc.c``
(Sec. 3, Eqs. 22-33, with the same readings: Gamma_i = 1 + s_i, the
isotropic stencils, ghost rows mirrored for phi and mu and extrapolated for
p at walls, halfway bounce-back with the moving-wall term), written as
whole-array torch operations, and its forward is pinned to ``orc.c`` by
``tests/test_torch_step.py``.  It shares no code with the CUDA path.

Parameters that the gradients are taken with respect to (the mobility M
and the surface tension sigma) enter as torch scalars: kappa, beta are
linear in sigma (Eqs. 3-4 solved), alpha and gamma * lambda linear in M
(Eq. 33, lambda = M).
"""
from __future__ import annotations

import numpy as np
import torch

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
WT = [4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
CS2 = 1.0 / 3.0


class TorchStep:
    """One domain; fields are [ny, nx] FP64 tensors, populations [9, ny, nx]."""

    def __init__(self, p: dict):
        self.p = dict(p)
        self.nx, self.ny = p["nx"], p["ny"]
        self.wall = p.get("bc_y", 0) == 1
        d = p["phi_A"] - p["phi_B"]
        self.dphi = d
        self.phibar = 0.5 * (p["phi_A"] + p["phi_B"])
        self.drho = (p["rho_A"] - p["rho_B"]) / d
        self.gamma = (p["rho_A"] - p["rho_B"]) / (p["rho_B"] * p["phi_A"] - p["rho_A"] * p["phi_B"])
        # per unit sigma / unit M
        self.kappa1 = 3.0 * p["W"] / (2.0 * d * d)
        self.beta1 = 12.0 / (p["W"] * d ** 4)
        self.alpha1 = 1.0 / (CS2 * (p["tau_g"] - 0.5))
        ny, nx = self.ny, self.nx
        yy = np.arange(ny)
        # neighbour rows: mirror (phi, mu) and the pair used to extrapolate p
        self.rows_m, self.rows_e = {}, {}
        for cy in (-1, 0, 1):
            r = yy + cy
            if self.wall:
                m = np.where(r < 0, -r - 1, np.where(r >= ny, 2 * ny - 1 - r, r))
                a = np.where(r < 0, 0, np.where(r >= ny, ny - 1, r))
                b = np.where(r < 0, 1, np.where(r >= ny, ny - 2, r))
                ca = np.where((r < 0) | (r >= ny), 2.0, 1.0)
                cb = np.where((r < 0) | (r >= ny), -1.0, 0.0)
            else:
                m = r % ny
                a, b, ca, cb = m, m, np.ones(ny), np.zeros(ny)
            self.rows_m[cy] = torch.as_tensor(m)
            self.rows_e[cy] = (torch.as_tensor(a), torch.as_tensor(b),
                               torch.as_tensor(ca)[:, None], torch.as_tensor(cb)[:, None])

    # ------------------------------------------------------------ stencils
    def _nb(self, v, cx, cy, extrap=False):
        """v at (x + cx, y + cy) with periodic x and the y ghost rule."""
        v = torch.roll(v, shifts=-cx, dims=1)
        if not extrap:
            return v[self.rows_m[cy]]
        a, b, ca, cb = self.rows_e[cy]
        return ca * v[a] + cb * v[b]

    def grad(self, v, extrap=False):
        gx = 0.0
        gy = 0.0
        for i in range(1, 9):
            n = self._nb(v, CX[i], CY[i], extrap)
            gx = gx + WT[i] * CX[i] * n
            gy = gy + WT[i] * CY[i] * n
        return gx / CS2, gy / CS2

    def lap(self, v):
        acc = 0.0
        for i in range(1, 9):
            acc = acc + WT[i] * (self._nb(v, CX[i], CY[i]) - v)
        return 2.0 * acc / CS2

    # ---------------------------------------------------------- the model
    def mu(self, phi, sigma):
        p = self.p
        dpsi = 4.0 * self.beta1 * sigma * (phi - p["phi_A"]) * (phi - p["phi_B"]) * (phi - self.phibar)
        return dpsi - self.kappa1 * sigma * self.lap(phi)

    def init(self, phi0, M, sigma):
        """Equilibrium initial state at p = 0, u = 0 (f = 0, g = H_i)."""
        mu = self.mu(phi0, sigma)
        amu = self.alpha1 * M * mu
        g = torch.stack([phi0 - (1.0 - WT[0]) * amu] + [WT[i] * amu for i in range(1, 9)])
        f = torch.zeros_like(g)
        return f, g

    def step(self, f, g, M, sigma):
        p = self.p
        phi = g.sum(0)
        rho = p["rho_B"] + (phi - p["phi_B"]) * self.drho
        mu = self.mu(phi, sigma)
        gphx, gphy = self.grad(phi)
        grhx, grhy = self.drho * gphx, self.drho * gphy
        gmux, gmuy = self.grad(mu)
        lmu = self.lap(mu)
        Fx = -phi * gmux
        Fy = -phi * gmuy - (rho - p["rho_ref"]) * p["gravity"]
        jx = sum(CX[i] * f[i] for i in range(9))
        jy = sum(CY[i] * f[i] for i in range(9))
        ux = (jx + 0.5 * CS2 * Fx) / (CS2 * rho)
        uy = (jy + 0.5 * CS2 * Fy) / (CS2 * rho)
        gl = self.gamma * M
        pr = f.sum(0) + 0.5 * CS2 * (ux * grhx + uy * grhy - gl * rho * lmu)
        gpx, gpy = self.grad(pr, extrap=True)
        amu = self.alpha1 * M * mu
        uu = ux * ux + uy * uy
        tf, tg = p["tau_f"], p["tau_g"]
        fs, gs = [], []
        for i in range(9):
            cu = CX[i] * ux + CY[i] * uy
            si = cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2)
            Gam = 1.0 + si
            H = phi - (1.0 - WT[0]) * amu if i == 0 else WT[i] * amu
            feq = WT[i] * (pr + CS2 * rho * si)
            geq = H + WT[i] * phi * si
            ex, ey = CX[i] - ux, CY[i] - uy
            Fi = (ex * (WT[i] * Gam * Fx + WT[i] * si * CS2 * grhx)
                  + ey * (WT[i] * Gam * Fy + WT[i] * si * CS2 * grhy)
                  - WT[i] * CS2 * rho * gl * lmu)
            Gi = -(phi / (CS2 * rho)) * (ex * (gpx - Fx) + ey * (gpy - Fy)) * WT[i] * Gam
            fs.append(f[i] - (f[i] - feq) / tf + (1.0 - 0.5 / tf) * Fi)
            gs.append(g[i] - (g[i] - geq) / tg + (1.0 - 0.5 / tg) * Gi)
        return self._stream(fs, gs, rho, phi)

    def _stream(self, fs, gs, rho, phi):
        """f_i(y) = f*_i(y - c_i); a population whose upstream cell lies beyond
        a wall is the bounced f*_opp(y) minus twice its equilibrium's linear
        term at the wall velocity."""
        ny = self.ny
        yy = torch.arange(ny)[:, None]
        out_f, out_g = [], []
        p = self.p
        for i in range(9):
            up = torch.roll(fs[i], shifts=(CY[i], CX[i]), dims=(0, 1))
            ug = torch.roll(gs[i], shifts=(CY[i], CX[i]), dims=(0, 1))
            if self.wall and CY[i] != 0:
                src_row = yy - CY[i]
                bounced = (src_row < 0) | (src_row >= ny)
                o = OPP[i]
                # population o at y leaves through the wall it faces
                uw = p["u_wall_bottom"] if CY[o] < 0 else p["u_wall_top"]
                cu = CX[o] * uw
                bf = fs[o] - 2.0 * WT[o] * rho * cu
                bg = gs[o] - 2.0 * WT[o] * phi * cu / CS2
                up = torch.where(bounced, bf, up)
                ug = torch.where(bounced, bg, ug)
            out_f.append(up)
            out_g.append(ug)
        return torch.stack(out_f), torch.stack(out_g)

    def fields(self, f, g, M, sigma):
        """phi, u, p of a state (as orc_fields)."""
        p = self.p
        phi = g.sum(0)
        rho = p["rho_B"] + (phi - p["phi_B"]) * self.drho
        mu = self.mu(phi, sigma)
        gphx, gphy = self.grad(phi)
        gmux, gmuy = self.grad(mu)
        lmu = self.lap(mu)
        Fx = -phi * gmux
        Fy = -phi * gmuy - (rho - p["rho_ref"]) * p["gravity"]
        jx = sum(CX[i] * f[i] for i in range(9))
        jy = sum(CY[i] * f[i] for i in range(9))
        ux = (jx + 0.5 * CS2 * Fx) / (CS2 * rho)
        uy = (jy + 0.5 * CS2 * Fy) / (CS2 * rho)
        pr = f.sum(0) + 0.5 * CS2 * (self.drho * (ux * gphx + uy * gphy) - self.gamma * M * rho * lmu)
        return {"phi": phi, "rho": rho, "ux": ux, "uy": uy, "p": pr, "mu": mu}

    def rollout_loss(self, phi0, M, sigma, steps, target):
        f, g = self.init(phi0, M, sigma)
        for _ in range(steps):
            f, g = self.step(f, g, M, sigma)
        return ((g.sum(0) - target) ** 2).sum()
