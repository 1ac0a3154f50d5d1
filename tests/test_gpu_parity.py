"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.

Tolerances: FP64 path within 1e-12 relative to the field's maximum
magnitude; FP32 path within 1e-5 max-abs on phi and u (and within the
arithmetic's reach on p and rho).  Cases span several 32 x 16 tiles with
ragged tails, grids smaller than a tile, walls (moving, with gravity) and
zero steps.  Full-size grids are checked on sampled cells: after k steps a
cell depends only on the initial state within 4k + 1 cells (the stencil
chain phi -> mu -> p -> grad p reaches 3 cells, streaming 1, the initial
mu 1), so the oracle run on a periodic window of the initial field around
the sample reproduces that cell exactly.
"""
import numpy as np
import pytest

import oracle
from helpers import check64, oracle_spread, same_result
from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "rho", "p", "ux", "uy", "mu")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm as L
    build.build()
    return L


def _run_gpu(L, p, phi, ux, uy, steps, dtype):
    s = L.Sim(p, dtype)
    s.init_phi(phi, ux, uy)
    s.step(steps)
    out = {k: v.double().cpu().numpy() for k, v in s.fields().items()}
    m = s.mass()
    s.close()
    return out, m


def _run_orc(p, phi, ux, uy, steps):
    o = oracle.Oracle(p)
    o.init_phi(phi, ux, uy)
    o.step(steps)
    return o.fields(), o.mass(), o


# Grids with nx % 8 == 0 run the strip kernel; the others the tile kernel.
CASES = [
    ("tiny5x5", lambda: W.small_case(5, 5, seed=1), 10),
    ("odd6x7", lambda: W.small_case(6, 7, seed=2), 10),
    ("ragged37x29", lambda: W.small_case(37, 29, seed=3), 25),
    ("tiles70x45", lambda: W.small_case(70, 45, seed=4), 25),
    ("walls37x29", lambda: W.small_case(37, 29, seed=5, walls=True, gravity=2e-5, u_wall=0.02), 25),
    ("walls9x5", lambda: W.small_case(9, 5, seed=6, walls=True, gravity=1e-5, u_wall=-0.01), 15),
    ("walls33x34", lambda: W.small_case(33, 34, seed=7, walls=True, gravity=1e-5, u_wall=0.01), 20),
    ("droplet64", lambda: W.droplet64() + (None, None), 50),
    ("zero_steps", lambda: W.small_case(40, 24, seed=8), 0),
    ("strip32x29", lambda: W.small_case(32, 29, seed=14), 20),
    ("strip136x37", lambda: W.small_case(136, 37, seed=15), 20),
    ("strip_walls24x5", lambda: W.small_case(24, 5, seed=16, walls=True, gravity=1e-5, u_wall=0.02), 15),
    ("strip_walls200x45", lambda: W.small_case(200, 45, seed=17, walls=True, gravity=2e-5, u_wall=-0.01), 25),
    ("strip_walls8x70", lambda: W.small_case(8, 70, seed=18, walls=True, gravity=1e-5, u_wall=0.01), 20),
    # 368 columns: strips 1 and 2 lie inside the level and take their rows
    # by tensor tiles (FP32); strips 0 and 3 wrap and copy by chunks
    ("tiles368x45", lambda: W.small_case(368, 45, seed=19), 20),
    ("tiles_walls368x29", lambda: W.small_case(368, 29, seed=20, walls=True, gravity=1e-5, u_wall=0.01), 20),
]


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_f64_matches_oracle(lbm, name, make, steps):
    p, phi, ux, uy = make()
    g, gm = _run_gpu(lbm, p, phi, ux, uy, steps, "f64")
    o, om, _ = _run_orc(p, phi, ux, uy, steps)
    check64(g, o, oracle_spread(p, phi, ux, uy, steps, o), name)
    assert abs(gm[0] - om[0]) <= 1e-12 * abs(om[0])
    assert abs(gm[1] - om[1]) <= 1e-12 * np.abs(phi).sum()


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_f32_matches_oracle(lbm, name, make, steps):
    p, phi, ux, uy = make()
    g, _ = _run_gpu(lbm, p, phi, ux, uy, steps, "f32")
    o, _, _ = _run_orc(p, phi, ux, uy, steps)
    for k in ("phi", "ux", "uy"):
        err = np.abs(g[k] - o[k]).max()
        assert err <= 1e-5, f"{name}: {k} max-abs error {err:.3e}"
    assert np.abs(g["rho"] - o["rho"]).max() <= 1e-5
    assert np.abs(g["p"] - o["p"]).max() <= 1e-5 * max(1.0, np.abs(o["p"]).max())


def test_f64_populations_match_oracle(lbm):
    """The FP64 state (layout f_0..8, g_0..8, slot stride NS) equals the
    oracle's populations cell by cell."""
    p, phi, ux, uy = W.small_case(37, 29, seed=11, walls=True, gravity=1e-5, u_wall=0.01)
    s = lbm.Sim(p, "f64")
    s.init_phi(phi, ux, uy)
    s.step(13)
    buf, step = s.get_state()
    assert step == 13
    N = 37 * 29
    NS = (N + 127) // 128 * 128
    a = buf.cpu().numpy().view(np.float64).reshape(18, NS)[:, :N].reshape(18, 29, 37)
    o = oracle.Oracle(p)
    o.init_phi(phi, ux, uy)
    o.step(13)
    f, g = o.pops()
    ref = np.concatenate([f, g])
    err = np.abs(a - ref).max() / np.abs(ref).max()
    assert err <= 1e-12


def _window_check(L, p, phi, dtype, steps, samples, tol_phi_u, rel64=None):
    """Full-size GPU run checked at sampled cells against the oracle on a
    periodic window (half-width h > 4 steps + 1) around each sample.  FP64:
    max error over the samples within rel64 of the largest sampled oracle
    magnitude of that field; FP32: max-abs bound on phi and u."""
    ny, nx = phi.shape
    s = L.Sim(p, dtype)
    s.init_phi(phi)
    s.step(steps)
    g = {k: v.double().cpu().numpy() for k, v in s.fields().items()}
    s.close()
    h = 4 * steps + 1 + 8
    got = {k: [] for k in ("phi", "ux", "uy", "p")}
    ref = {k: [] for k in got}
    for (yy, xx) in samples:
        ys = np.arange(yy - h, yy + h + 1) % ny
        xs = np.arange(xx - h, xx + h + 1) % nx
        win = phi[np.ix_(ys, xs)]
        q = dict(p, nx=2 * h + 1, ny=2 * h + 1)
        o = oracle.Oracle(q)
        o.init_phi(win)
        o.step(steps)
        of = o.fields()
        for k in got:
            got[k].append(g[k][yy, xx])
            ref[k].append(of[k][h, h])
    for k in got:
        a, b = np.array(got[k]), np.array(ref[k])
        err = np.abs(a - b).max()
        if rel64 is not None:
            assert err <= rel64 * np.abs(b).max(), (k, err, np.abs(b).max())
        elif k in ("phi", "ux", "uy"):
            assert err <= tol_phi_u, (k, err)


def _samples(nx, ny, seed, n=12):
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (ny - 1, nx - 1), (0, nx - 1), (ny - 1, 0), (ny // 2, nx // 2)]
    pts += [(int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(n)]
    return pts


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_full_size_precision_workload_sampled(lbm, dtype):
    """4096 x 4096, 512 droplets, rho_A/rho_B = 100: the benchmark workload,
    in the benchmark's launch configuration, 3 steps, sampled cells (some on
    droplet interfaces, some on the periodic seams)."""
    p, phi = W.precision()
    # interface cells: where |phi| < 0.5
    rng = np.random.default_rng(3)
    iy, ix = np.nonzero(np.abs(phi) < 0.5)
    pick = rng.choice(len(iy), 8, replace=False)
    samples = _samples(4096, 4096, 5) + [(int(iy[i]), int(ix[i])) for i in pick]
    _window_check(lbm, p, phi, dtype, 3, samples, 1e-5, rel64=1e-12 if dtype == "f64" else None)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_rayleigh_taylor(lbm, dtype):
    """256 x 1024 with walls and gravity, element by element, 20 steps."""
    p, phi = W.rayleigh_taylor()
    g, gm = _run_gpu(lbm, p, phi, None, None, 20, dtype)
    o, om, _ = _run_orc(p, phi, None, None, 20)
    if dtype == "f64":
        check64(g, o, oracle_spread(p, phi, None, None, 20, o), "rayleigh_taylor")
    else:
        for k in ("phi", "ux", "uy"):
            assert np.abs(g[k] - o[k]).max() <= 1e-5, k


def test_conservation_long_f64(lbm):
    p, phi, ux, uy = W.small_case(48, 40, seed=9, walls=True, gravity=1e-5, u_wall=0.01)
    s = lbm.Sim(p, "f64")
    s.init_phi(phi, ux, uy)
    m0, t0 = s.mass()
    s.step(2000)
    m1, t1 = s.mass()
    assert abs(m1 - m0) <= 1e-13 * m0
    assert abs(t1 - t0) <= 1e-13 * np.abs(phi).sum()


@pytest.mark.parametrize("shape", [(70, 45), (64, 48)])
def test_resume_is_bit_identical(lbm, shape):
    p, phi, ux, uy = W.small_case(shape[0], shape[1], seed=10)
    for dtype in ("f32", "f16s", "bf16s", "f64"):
        a = lbm.Sim(p, dtype)
        a.init_phi(phi, ux, uy)
        a.step(7)
        buf, step = a.get_state()
        a.step(9)
        fa = {k: v.cpu().numpy() for k, v in a.fields().items()}
        b = lbm.Sim(p, dtype)
        b.set_state(buf, step)
        b.step(9)
        fb = {k: v.cpu().numpy() for k, v in b.fields().items()}
        assert b.step_count == 16
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), (dtype, k)


@pytest.mark.parametrize("shape", [(70, 45), (64, 48)])
def test_runs_are_deterministic(lbm, shape):
    p, phi, ux, uy = W.small_case(shape[0], shape[1], seed=12)
    outs = []
    for _ in range(2):
        s = lbm.Sim(p, "f32")
        s.init_phi(phi, ux, uy)
        s.step(11)
        outs.append((s.fields()["phi"].cpu().numpy(), s.mass()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_host_buffers_match_device_path(lbm):
    p, phi, ux, uy = W.small_case(37, 29, seed=13)
    r = lbm.run_host(p, phi, 9, "f32", ux, uy, names=("phi", "ux", "uy", "p"))
    s = lbm.Sim(p, "f32")
    s.init_phi(phi, ux, uy)
    s.step(9)
    d = {k: v.cpu().numpy() for k, v in s.fields().items()}
    for k in ("phi", "ux", "uy", "p"):
        assert np.array_equal(r.fields[k], d[k]), k


def test_laplace_diagnostic_matches_oracle(lbm):
    p, phi = W.droplet64()
    s = lbm.Sim(p, "f64")
    s.init_phi(phi)
    s.step(200)
    dP, Re = s.laplace(32.0, 32.0, 16.0)
    o = oracle.Oracle(p)
    o.init_phi(phi)
    o.step(200)
    odP, oRe = o.laplace(32.0, 32.0, 16.0)
    assert abs(dP - odP) <= 1e-10 * abs(odP)
    assert abs(Re - oRe) <= 1e-12 * oRe


@pytest.mark.parametrize("dtype,tol", [("f16s", 2e-3), ("bf16s", 3e-2)])
def test_16bit_storage_error_and_conservation(lbm, dtype, tol):
    """16-bit storage: phi and u stay close to the FP64 oracle (the bound is
    the measured error, stated in the design notes), and sum phi is
    conserved to FP32 rounding because g_0 absorbs the rounding of the
    other populations."""
    p, phi = W.droplet64()
    g, gm = _run_gpu(lbm, p, phi, None, None, 200, dtype)
    o, om, _ = _run_orc(p, phi, None, None, 200)
    assert np.abs(g["phi"] - o["phi"]).max() <= tol
    assert np.abs(g["ux"] - o["ux"]).max() <= tol * 0.1
    s = lbm.Sim(p, dtype)
    s.init_phi(phi)
    m0, t0 = s.mass()
    s.step(500)
    m1, t1 = s.mass()
    assert abs(t1 - t0) <= 2e-5 * np.abs(phi).sum()


@pytest.mark.parametrize("dtype,tol", [("f16s", 2e-3), ("bf16s", 3e-2)])
def test_16bit_tensor_tile_strips_match_oracle(lbm, dtype, tol):
    """Raw 16-bit storage on a 368-column walled grid, whose two middle
    strips load their rows as tensor tiles: phi and u within the 16-bit
    bounds of the FP64 oracle, sum phi conserved to FP32 rounding."""
    p, phi, ux, uy = W.small_case(368, 45, seed=22, walls=True, gravity=1e-5, u_wall=0.01)
    g, gm = _run_gpu(lbm, p, phi, ux, uy, 60, dtype)
    o, om, _ = _run_orc(p, phi, ux, uy, 60)
    assert np.abs(g["phi"] - o["phi"]).max() <= tol
    assert max(np.abs(g["ux"] - o["ux"]).max(), np.abs(g["uy"] - o["uy"]).max()) <= tol * 0.1
    assert abs(gm[1] - om[1]) <= 2e-5 * np.abs(phi).sum()


def test_errors_surface_through_the_abi(lbm):
    p, phi = W.droplet64()
    s = lbm.Sim(p, "f32")
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.status == -5
    s.init_phi(phi)
    with pytest.raises(lbm.LBMError):
        s.step(-1)
    bad = phi.copy()
    bad[3, 4] = np.nan
    s.init_phi(bad)
    s.step(2)
    with pytest.raises(lbm.LBMError) as e:
        s.mass()
    assert e.value.status == -3


@pytest.mark.parametrize("dtype", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("walls", [False, True])
def test_tensor_tile_rows_equal_chunk_copies(lbm, walls, dtype):
    """Single domains in FP32 and raw 16-bit storage stage the rows of
    strips that lie inside the level by TMA tensor tiles (16-bit: the g_0
    floats and the half slots from three maps); the batched form copies
    every row by 16-byte chunks.  Same rows in shared memory and the same
    per-cell arithmetic, so the two agree (helpers.same_result: FP32 to
    rounding, since different kernels may contract multiply-adds
    differently)."""
    p, phi, ux, uy = W.small_case(368, 61, seed=21, walls=walls, gravity=1e-5 if walls else 0.0,
                                  u_wall=0.01 if walls else 0.0)
    s = lbm.Sim(p, dtype)
    s.init_phi(phi)
    s.step(9)
    a = {k: v.cpu().numpy() for k, v in s.fields(("phi", "ux", "uy", "p")).items()}
    sm = s.mass()
    s.close()
    b = lbm.Batch([p], dtype)
    b.init_phi([phi])
    b.step(9)
    g = b.fields()[0]
    for k in a:
        same_result(a[k], g[k].cpu().numpy(), dtype, k)
    assert abs(b.mass()[0][0] - sm[0]) <= 1e-9 * abs(sm[0])
    b.close()
