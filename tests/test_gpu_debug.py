"""The LBM_DEBUG build (liblbm_debug.so): the same kernels with every
population and field index of the single-domain path bounds-checked.  On
tiny, ragged and walled grids, in every storage form, it runs clean (no
check fails, so lbm_mass returns LBM_OK) and gives the results of the
release build: bit for bit in FP64, which is built without contracted
multiply-adds; within FP32 rounding in the forms with FP32 arithmetic,
where the compiler is free to contract a product and a sum into one FMA
and the extra checks change where it does."""
import numpy as np
import pytest

from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm
    build.build()
    build.build(debug=True)
    return lbm


CASES = [
    ("tiny5x5", lambda: W.small_case(5, 5, seed=1), 10),               # tile kernel
    ("odd6x7", lambda: W.small_case(6, 7, seed=2), 10),
    ("walls37x29", lambda: W.small_case(37, 29, seed=5, walls=True, gravity=2e-5, u_wall=0.02), 15),
    ("strip_walls24x5", lambda: W.small_case(24, 5, seed=16, walls=True, gravity=1e-5, u_wall=0.02), 15),
    ("strip_walls8x70", lambda: W.small_case(8, 70, seed=18, walls=True, gravity=1e-5, u_wall=0.01), 15),
    ("strip136x37", lambda: W.small_case(136, 37, seed=15), 15),           # strip kernel, ragged strip
    ("strip_walls200x45", lambda: W.small_case(200, 45, seed=17, walls=True, gravity=2e-5, u_wall=-0.01), 10),
]


def _run(L, p, phi, ux, uy, steps, dtype, debug):
    s = L.Sim(p, dtype, debug=debug)
    s.init_phi(phi, ux, uy)
    s.step(steps)
    m = s.mass()  # LBM_ERR_STATE if an index check failed
    f = {k: v.cpu().numpy() for k, v in s.fields().items()}
    s.close()
    return f, m


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s", "f16d"])
def test_debug_build_runs_clean_and_matches_release(L, name, make, steps, dtype):
    p, phi, ux, uy = make()
    if dtype == "f16d" and p["nx"] % 8 != 0:
        pytest.skip("the deviation storage needs nx a multiple of 8")
    rel, m_rel = _run(L, p, phi, ux, uy, steps, dtype, False)
    dbg, m_dbg = _run(L, p, phi, ux, uy, steps, dtype, True)
    for k in rel:
        if dtype == "f64":
            assert np.array_equal(rel[k], dbg[k]), (name, dtype, k)
        else:
            err = float(np.abs(rel[k].astype(np.float64) - dbg[k]).max())
            assert err <= 1e-5 * max(1.0, float(np.abs(rel[k]).max())), (name, dtype, k, err)
    if dtype == "f64":
        assert m_rel == m_dbg
    else:
        assert abs(m_rel[0] - m_dbg[0]) <= 1e-6 * abs(m_rel[0])
