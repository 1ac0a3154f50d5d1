"""The y-slab decomposition (lbm_slabs_*) against the whole-domain step.

A domain split into slabs that step separately and exchange ghost rows on
the device must reproduce the whole-domain state: every cell runs the same
kernel body, and the exchange only moves populations.  Bit for bit in FP64
and the 16-bit forms; within FP32 rounding in FP32, where the slab kernel
and the whole-domain kernel (which stages interior rows by tensor tiles)
are compiled separately and nvcc may contract multiply-adds differently.  The
cases cover periodic and wall-bounded domains (moving walls, gravity), even
and uneven splits, the smallest slab (3 rows), one slab across the periodic
wrap, interior strips (fast push path) and edge strips, and every storage
form.
"""
import numpy as np
import pytest

from helpers import same_result
from paper_1507_03521_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm as L
    build.build()
    return L


def _slots(buf, dtype, n):
    """The 18 population slots of a whole-domain level (cells 0..n-1 each),
    as raw bytes: (f_0..f_8, g_0..g_8)."""
    ns = (n + 127) // 128 * 128
    b = buf.cpu().numpy()
    if dtype in ("f32", "f64"):
        e = 8 if dtype == "f64" else 4
        return [b[q * ns * e:(q * ns + n) * e] for q in range(18)]
    g0 = b[:n * 4]
    half = [b[ns * 4 + s * ns * 2: ns * 4 + (s * ns + n) * 2] for s in range(17)]
    return half[:9] + [g0] + half[9:]


def _compare(L, p, phi, ux, uy, dtype, steps, **kw):
    a = L.Sim(p, dtype)
    a.init_phi(phi, ux, uy)
    s0, _ = a.get_state()
    s0 = s0.clone()
    a.step(steps)
    ref, _ = a.get_state()
    s = L.Slabs(p, dtype, **kw)
    s.scatter(s0, 0)
    s.step(steps)
    got, step = s.gather()
    assert step == steps and s.step_count == steps
    n = p["nx"] * p["ny"]
    for q, (x, y) in enumerate(zip(_slots(ref, dtype, n), _slots(got, dtype, n))):
        if dtype == "f32":
            same_result(x.view(np.float32), y.view(np.float32), dtype, (q, kw))
        else:
            assert np.array_equal(x, y), (dtype, q, kw)
    s.close()
    a.close()


@pytest.mark.parametrize("dtype", ["f32", "f16s", "bf16s", "f64"])
@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("split", [dict(n_slabs=1), dict(n_slabs=2), dict(n_slabs=3),
                                   dict(row_starts=[0, 3, 20, 23])])
def test_slabs_bit_identical_to_whole_domain(lbm, dtype, walls, split):
    p, phi, ux, uy = W.small_case(384, 45, seed=31, walls=walls, gravity=2e-5 if walls else 0.0,
                                  u_wall=0.02 if walls else 0.0)
    _compare(lbm, p, phi, ux, uy, dtype, 9, **split)


def test_slabs_narrow_domain_many_slabs(lbm):
    """One 64-column strip (edge pushes only), 8 slabs of 3 to 5 rows."""
    p, phi, ux, uy = W.small_case(64, 29, seed=32)
    _compare(lbm, p, phi, ux, uy, "f32", 13, row_starts=[0, 3, 7, 10, 14, 17, 21, 25])


def test_slabs_long_run_bench_shape(lbm):
    """A 4-slab split of a 1024 x 512 multi-droplet field at the bench's
    density ratio, 40 steps."""
    p, phi = W.precision(n=512, n_drops=8)
    p = dict(p, nx=1024)
    phi = np.concatenate([phi, phi[:, ::-1]], axis=1)
    _compare(lbm, p, phi, None, None, "f32", 40, n_slabs=4)


def test_slabs_reject_bad_splits(lbm):
    p, phi, _, _ = W.small_case(64, 29, seed=33)
    with pytest.raises(lbm.LBMError):
        lbm.Slabs(p, "f32", row_starts=[0, 2, 10])       # a slab of 2 rows
    with pytest.raises(lbm.LBMError):
        lbm.Slabs(p, "f32", row_starts=[1, 10, 20])      # does not start at row 0
    with pytest.raises(lbm.LBMError):
        lbm.Slabs(dict(p, nx=60), "f32", n_slabs=2)      # nx not a multiple of 8
    with pytest.raises(lbm.LBMError):
        lbm.Slabs(p, "f32", n_slabs=10)                  # 29 rows cannot hold 10 slabs
