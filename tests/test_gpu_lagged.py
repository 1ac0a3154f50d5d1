"""The lagged-grad-p variant on the GPU (k_strip_lag, and k_strip_lag_tma for
FP32 strips whose rows come as tensor tiles) against the oracle's
lagged variant, element by element: FP64 within the FP64 bar, FP32 within
1e-5 on phi and u; resume from a saved state (which carries the stored
pressure) is bit-identical; the variant is refused where it is not built."""
import numpy as np
import pytest

import oracle
from helpers import check64, oracle_spread
from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    dict(shape=(64, 48), seed=51),
    dict(shape=(48, 37), seed=52, walls=True, gravity=2e-5, u_wall=0.02),
    dict(shape=(264, 40), seed=53),
    dict(shape=(392, 29), seed=54, walls=True, gravity=-1e-5, u_wall=-0.01),
    dict(shape=(8, 70), seed=55),
]


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm
    build.build()
    return lbm


def _case(c):
    nx, ny = c["shape"]
    p, phi, ux, uy = W.small_case(nx, ny, seed=c["seed"], walls=c.get("walls", False),
                                  gravity=c.get("gravity", 0.0), u_wall=c.get("u_wall", 0.0))
    return dict(p, gradp_lag=1), phi, ux, uy


def _oracle(p, phi, ux, uy, steps):
    o = oracle.Oracle(p)
    o.init_phi(phi, ux, uy)
    o.step(steps)
    return o.fields()


@pytest.mark.parametrize("c", CASES, ids=lambda c: "x".join(map(str, c["shape"])))
def test_lagged_f64_matches_oracle(L, c):
    p, phi, ux, uy = _case(c)
    steps = 40
    ref = _oracle(p, phi, ux, uy, steps)
    s = L.Sim(p, "f64")
    s.init_phi(phi, ux, uy)
    s.step(steps)
    got = {k: v.cpu().numpy() for k, v in s.fields().items()}
    check64(got, ref, oracle_spread(p, phi, ux, uy, steps, ref), f"lagged {c['shape']}")


# 264 and 392 columns: the middle strips take their g and f rows as
# tensor tiles (k_strip_lag_tma), periodic and walled
@pytest.mark.parametrize("c", CASES[:4], ids=lambda c: "x".join(map(str, c["shape"])))
def test_lagged_f32_matches_oracle(L, c):
    p, phi, ux, uy = _case(c)
    steps = 40
    ref = _oracle(p, phi, ux, uy, steps)
    s = L.Sim(p, "f32")
    s.init_phi(phi, ux, uy)
    s.step(steps)
    got = {k: v.double().cpu().numpy() for k, v in s.fields().items()}
    for k in ("phi", "ux", "uy"):
        assert np.abs(got[k] - ref[k]).max() < 1e-5, k


def test_lagged_is_not_the_synchronous_step(L):
    p, phi, ux, uy = _case(CASES[0])
    out = []
    for lag in (0, 1):
        s = L.Sim(dict(p, gradp_lag=lag), "f64")
        s.init_phi(phi, ux, uy)
        s.step(20)
        out.append(s.fields(("phi",))["phi"].cpu().numpy())
    assert np.abs(out[0] - out[1]).max() > 1e-9


@pytest.mark.parametrize("dtype", ["f32", "f16s", "bf16s", "f64"])
def test_lagged_resume_bit_identical(L, dtype):
    p, phi, ux, uy = _case(CASES[1])
    a = L.Sim(p, dtype)
    a.init_phi(phi, ux, uy)
    a.step(6)
    buf, step = a.get_state()
    buf = buf.clone()
    a.step(9)
    fa = {k: v.cpu().numpy() for k, v in a.fields().items()}
    b = L.Sim(p, dtype)
    b.set_state(buf, step)
    b.step(9)
    fb = {k: v.cpu().numpy() for k, v in b.fields().items()}
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), (dtype, k)


@pytest.mark.parametrize("dtype,tol", [("f16s", 5e-4), ("bf16s", 5e-3)])
def test_lagged_16bit_forms(L, dtype, tol):
    p, phi, ux, uy = _case(CASES[2])
    ref = L.Sim(p, "f64")
    ref.init_phi(phi, ux, uy)
    ref.step(40)
    r = ref.fields(("phi",))["phi"].cpu().numpy()
    s = L.Sim(p, dtype)
    s.init_phi(phi, ux, uy)
    s.step(40)
    assert np.abs(s.fields(("phi",))["phi"].double().cpu().numpy() - r).max() < tol


def test_lagged_refused_where_not_built(L):
    p, phi, _, _ = W.small_case(60, 30, seed=56)
    with pytest.raises(L.LBMError):
        L.Sim(dict(p, gradp_lag=1), "f32")                 # nx not a multiple of 8
    q, _, _, _ = W.small_case(64, 30, seed=56)
    with pytest.raises(L.LBMError):
        L.Batch([dict(q, gradp_lag=1)], "f32")
    with pytest.raises(L.LBMError):
        L.Slabs(dict(q, gradp_lag=1), "f32", n_slabs=2)
    s = L.Sim(dict(q, gradp_lag=1), "f64")
    with pytest.raises(L.LBMError):
        s.adj_work()
