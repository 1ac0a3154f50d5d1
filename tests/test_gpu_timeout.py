"""The timeout path of the bounded waits, made to run out on purpose and
read back on the host; the GPU context stays usable.

FP32 single domains stage population rows by TMA tile loads that complete
on mbarriers, and every wait for one gives up after about a second.  The
test hook lbm_test_unfinished_tiles makes each load announce 16 bytes more
than it brings, so no wait can finish: the kernel sets the handle's error
word and its CTAs return; lbm_mass reports LBM_ERR_TIMEOUT.  Nothing
faults, traps or hangs.  Afterwards the same handle, re-initialised, steps
exactly as a fresh one."""
import time

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
    return lbm


def test_a_tile_wait_that_runs_out_reports_timeout(L):
    # 368 columns: the two middle strips take their rows by tile loads
    p, phi, ux, uy = W.small_case(368, 45, seed=23)
    s = L.Sim(p, "f32")
    s.init_phi(phi, ux, uy)
    s.test_unfinished_tiles(True)
    t0 = time.perf_counter()
    s.step(1)
    with pytest.raises(L.LBMError) as e:
        s.mass()
    elapsed = time.perf_counter() - t0
    assert e.value.status == -4, e.value
    assert elapsed < 30.0
    # the context and the handle are usable again
    s.test_unfinished_tiles(False)
    s.init_phi(phi, ux, uy)
    s.step(5)
    m = s.mass()
    got = {k: v.cpu().numpy() for k, v in s.fields(("phi", "ux", "uy", "p")).items()}
    s.close()
    ref = L.Sim(p, "f32")
    ref.init_phi(phi, ux, uy)
    ref.step(5)
    want = {k: v.cpu().numpy() for k, v in ref.fields(("phi", "ux", "uy", "p")).items()}
    assert ref.mass() == m
    ref.close()
    for k in got:
        assert np.array_equal(got[k], want[k]), k
