"""Pins of the oracle's isotropic finite-difference stencils (end of Sec. 3).

The paper only names an "isotropic central scheme".  The oracle reads it as
  grad chi = (1/c_s^2) sum_i w_i c_i chi(x + c_i),
  lap chi  = (2/c_s^2) sum_i w_i [chi(x + c_i) - chi(x)].
Pinned by their Fourier symbols on periodic grids (exact, closed form), by
exactness on low-order polynomials, and by the wall ghost rules compared
with numpy's own padding modes.
"""
import numpy as np
import pytest


def _mode(nx, ny, kx, ky, phase=0.3):
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    a, b = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    return a, b, np.cos(a * x + b * y + phase), np.sin(a * x + b * y + phase)


@pytest.mark.parametrize("kx,ky", [(1, 0), (0, 1), (1, 2), (3, -2), (5, 7), (8, 8)])
def test_fourier_symbols(orc, kx, ky):
    nx, ny = 24, 20
    a, b, c, s = _mode(nx, ny, kx, ky)
    gx, gy, lap = orc.stencils(c)
    lap_sym = 6.0 * ((2 / 9) * (np.cos(a) + np.cos(b)) + (1 / 9) * np.cos(a) * np.cos(b) - 5 / 9)
    gx_sym = 3.0 * np.sin(a) * (2 / 9 + (1 / 9) * np.cos(b))
    gy_sym = 3.0 * np.sin(b) * (2 / 9 + (1 / 9) * np.cos(a))
    # d/dx cos(theta) = -sin(theta) * a; the stencil gives -sin(theta) * gx_sym
    np.testing.assert_allclose(lap, lap_sym * c, rtol=0, atol=5e-14)
    np.testing.assert_allclose(gx, -gx_sym * s, rtol=0, atol=5e-14)
    np.testing.assert_allclose(gy, -gy_sym * s, rtol=0, atol=5e-14)


def test_symbols_consistent():
    # small-k limits of the symbols: lap -> -(a^2 + b^2), grad -> (a, b)
    for a, b in [(1e-3, 2e-3), (-3e-3, 1e-3)]:
        lap_sym = 6.0 * ((2 / 9) * (np.cos(a) + np.cos(b)) + (1 / 9) * np.cos(a) * np.cos(b) - 5 / 9)
        assert lap_sym == pytest.approx(-(a * a + b * b), rel=1e-5)
        assert 3.0 * np.sin(a) * (2 / 9 + np.cos(b) / 9) == pytest.approx(a, rel=1e-5)


def test_polynomial_exactness(orc):
    """Central gradient is exact on quadratics, the Laplacian on cubics,
    away from the periodic seam and the walls."""
    nx, ny = 16, 14
    x = np.arange(nx, dtype=float)[None, :] * np.ones((ny, 1))
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    q = 0.3 * x * x - 0.2 * x * y + 0.7 * y * y + 0.1 * x - 0.4 * y + 2.0
    cub = q + 0.01 * x ** 3 - 0.02 * x * x * y + 0.03 * y ** 3
    gx, gy, _ = orc.stencils(q, bc_y=1)
    _, _, lap = orc.stencils(cub, bc_y=1)
    sl = (slice(2, ny - 2), slice(2, nx - 2))
    np.testing.assert_allclose(gx[sl], (0.6 * x - 0.2 * y + 0.1)[sl], rtol=0, atol=1e-11)
    np.testing.assert_allclose(gy[sl], (-0.2 * x + 1.4 * y - 0.4)[sl], rtol=0, atol=1e-11)
    lap_exact = 0.6 + 1.4 + 0.06 * x - 0.04 * y + 0.18 * y
    np.testing.assert_allclose(lap[sl], lap_exact[sl], rtol=0, atol=1e-10)


def _ref_stencils(pad):
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ny, nx = pad.shape[0] - 2, pad.shape[1] - 2
    c = pad[1:-1, 1:-1]
    gx = np.zeros_like(c)
    gy = np.zeros_like(c)
    lap = np.zeros_like(c)
    for i in range(1, 9):
        v = pad[1 + cy[i]:1 + cy[i] + ny, 1 + cx[i]:1 + cx[i] + nx]
        gx += 3 * w[i] * cx[i] * v
        gy += 3 * w[i] * cy[i] * v
        lap += 6 * w[i] * (v - c)
    return gx, gy, lap


def test_wall_mirror_and_extrapolation(orc):
    rng = np.random.default_rng(11)
    chi = rng.standard_normal((9, 12))
    # phi, mu: even mirror about y = -1/2 and y = ny - 1/2 == numpy 'symmetric'
    pad = np.pad(chi, ((1, 1), (0, 0)), mode="symmetric")
    pad = np.pad(pad, ((0, 0), (1, 1)), mode="wrap")
    gx, gy, lap = orc.stencils(chi, bc_y=1)
    rgx, rgy, rlap = _ref_stencils(pad)
    np.testing.assert_allclose(gx, rgx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(gy, rgy, rtol=0, atol=1e-14)
    np.testing.assert_allclose(lap, rlap, rtol=0, atol=1e-13)
    # p: linear extrapolation across the wall == numpy 'reflect' with odd type
    pad = np.pad(chi, ((1, 1), (0, 0)), mode="reflect", reflect_type="odd")
    pad = np.pad(pad, ((0, 0), (1, 1)), mode="wrap")
    gx, gy, _ = orc.stencils(chi, bc_y=1, extrap=True)
    rgx, rgy, _ = _ref_stencils(pad)
    np.testing.assert_allclose(gx, rgx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(gy, rgy, rtol=0, atol=1e-14)
    # periodic == numpy 'wrap'
    pad = np.pad(chi, 1, mode="wrap")
    gx, gy, lap = orc.stencils(chi, bc_y=0)
    rgx, rgy, rlap = _ref_stencils(pad)
    np.testing.assert_allclose(gx, rgx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(lap, rlap, rtol=0, atol=1e-13)
