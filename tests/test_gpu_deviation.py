"""The 16-bit deviation storage (LBM_F16D, LBM_BF16D): populations stored as
their deviations from the rest equilibrium of the cell they sit on (Eqs.
24-27 at u = 0), FP32 arithmetic.

Against the FP64 oracle on the same seeded inputs, next to the raw 16-bit
storage (LBM_F16S, LBM_BF16S): within the raw forms' error bounds, and
smaller errors than the raw form for flows near rest; sum phi conserved to
FP32 rounding (g_0 absorbs the rounding of the others); a run resumes bit
for bit from a saved level; the forms it does not support are refused."""
import numpy as np
import pytest

import oracle
from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm
    build.build()
    return lbm


def _gpu(L, p, phi, ux, uy, steps, dtype):
    s = L.Sim(p, dtype)
    s.init_phi(phi, ux, uy)
    s.step(steps)
    out = {k: v.double().cpu().numpy() for k, v in s.fields().items()}
    s.close()
    return out


def _orc(p, phi, ux, uy, steps):
    o = oracle.Oracle(p)
    o.init_phi(phi, ux, uy)
    o.step(steps)
    return o.fields()


CASES = [
    ("droplet64", lambda: W.droplet64() + (None, None), 200),
    ("walls48x40", lambda: W.small_case(48, 40, seed=51, walls=True, gravity=1e-5, u_wall=0.01), 100),
    ("periodic64x37", lambda: W.small_case(64, 37, seed=52), 100),
]


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_deviation_storage_error_against_oracle(L, name, make, steps, kind):
    """Max-abs error against the FP64 oracle within the 16-bit bounds of
    the raw forms (FP16 2e-3, BF16 3e-2 on phi; a tenth of that on u).
    Near rest (the droplet, u0 = 0) the stored deviations are much smaller
    than the populations, and the deviation form is measured better on u
    (1.4-2x) and p (5-7x), phi within 5%.  The seeded small cases start
    from random velocities of 0.01, far from rest: there both forms store
    numbers of the same size and neither is better."""
    p, phi, ux, uy = make()
    ref = _orc(p, phi, ux, uy, steps)
    raw = _gpu(L, p, phi, ux, uy, steps, kind + "s")
    dev = _gpu(L, p, phi, ux, uy, steps, kind + "d")
    tol = {"f16": 2e-3, "bf16": 3e-2}[kind]
    e_raw = {k: float(np.abs(raw[k] - ref[k]).max()) for k in ("phi", "ux", "uy", "p")}
    e_dev = {k: float(np.abs(dev[k] - ref[k]).max()) for k in ("phi", "ux", "uy", "p")}
    print(f"DEV {name} {kind}: raw {e_raw} deviation {e_dev}")
    assert e_dev["phi"] <= tol and max(e_dev["ux"], e_dev["uy"]) <= 0.1 * tol
    if name == "droplet64":
        assert e_dev["p"] <= 0.5 * e_raw["p"]
        assert max(e_dev["ux"], e_dev["uy"]) <= max(e_raw["ux"], e_raw["uy"])
        assert e_dev["phi"] <= 1.1 * e_raw["phi"]


@pytest.mark.parametrize("dtype", ["f16d", "bf16d"])
def test_deviation_storage_conserves_phi(L, dtype):
    p, phi, ux, uy = W.small_case(64, 48, seed=53, walls=True, gravity=1e-5, u_wall=0.01)
    s = L.Sim(p, dtype)
    s.init_phi(phi, ux, uy)
    m0, t0 = s.mass()
    s.step(500)
    m1, t1 = s.mass()
    assert abs(t1 - t0) <= 2e-5 * np.abs(phi).sum()
    assert abs(m1 - m0) <= 2e-5 * m0
    s.close()


@pytest.mark.parametrize("dtype", ["f16d", "bf16d"])
def test_deviation_storage_resumes_bit_for_bit(L, dtype):
    p, phi, ux, uy = W.small_case(72, 45, seed=54)
    a = L.Sim(p, dtype)
    a.init_phi(phi, ux, uy)
    a.step(7)
    buf, step = a.get_state()
    a.step(9)
    fa = {k: v.cpu().numpy() for k, v in a.fields().items()}
    b = L.Sim(p, dtype)
    b.set_state(buf, step)
    b.step(9)
    fb = {k: v.cpu().numpy() for k, v in b.fields().items()}
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_deviation_storage_refuses_unsupported_forms(L):
    p, phi, _, _ = W.small_case(36, 20, seed=55)
    with pytest.raises(L.LBMError):
        L.Sim(p, "f16d")  # nx not a multiple of 8
    q, _ = W.droplet64()
    with pytest.raises(L.LBMError):
        L.Sim(dict(q, gradp_lag=1), "bf16d")
    with pytest.raises(L.LBMError):
        L.Batch([q, q], "f16d")
    with pytest.raises(L.LBMError):
        L.Slabs(q, "bf16d", n_slabs=2)


def test_deviation_storage_large_grid_sampled(L):
    """1024 x 1024, 32 droplets, rho_A/rho_B = 100 (the precision workload
    at a quarter of its side, at rest), 100 steps: the deviation forms
    against the FP32 path, which the FP32 parity tests tie to the oracle;
    the deviation form stays closer to FP32 than the raw form (FP16: 1.5x
    on phi, u at the FP32 level in both forms; BF16: 2x on both)."""
    p, phi = W.precision(n=1024, n_drops=32)
    f32 = _gpu(L, p, phi, None, None, 100, "f32")
    for kind in ("f16", "bf16"):
        raw = _gpu(L, p, phi, None, None, 100, kind + "s")
        dev = _gpu(L, p, phi, None, None, 100, kind + "d")
        for k in ("phi", "ux", "uy"):
            er = float(np.abs(raw[k] - f32[k]).max())
            ed = float(np.abs(dev[k] - f32[k]).max())
            print(f"DEV1024 {kind} {k}: raw {er:.3e} deviation {ed:.3e}")
            # FP16 u: both forms sit at the FP32 level here (within 3% of
            # each other over several runs); every other field and BF16
            # measured 1.5-2x better with deviations
            slack = 1.1 if (kind == "f16" and k != "phi") else 1.0
            assert ed <= slack * er, (kind, k, ed, er)
