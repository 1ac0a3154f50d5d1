"""GPU test of lbm_mass_noalloc, the mass diagnostic for callers that cannot
allocate device memory (a fixed device-memory budget owned by someone else,
a plug-in that must not grow the device footprint, a loop that cannot take
cudaMalloc's implicit synchronisation).  It runs with no handle and no work
buffer, on scratch that lives inside the library.

Checked through the C ABI against lbm_mass, the entry point that uses a
caller-bound work buffer: the two reduce in different orders, so they agree
to FP64 rounding (the 1e-12 relative bound of the other mass tests).  Four
calls in a row, largest grid first, so a later call on a smaller grid would
expose stale partial sums left by the earlier one; the first grid (1500 x
1400) spans several reduction blocks with a partial last block, and the
four calls cover every storage form.  This file is collected last so that
a run stopping at the first failure has run every other test.
"""
import ctypes

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
    lbm.load()
    return lbm


def _noalloc(L, params, dtype, level_ptr, stream_ptr):
    lib = L.load()
    cp = L.make_params(params, dtype)
    m, t = ctypes.c_double(), ctypes.c_double()
    st = lib.lbm_mass_noalloc(ctypes.byref(cp), ctypes.c_void_p(level_ptr),
                              ctypes.c_void_p(stream_ptr), ctypes.byref(m), ctypes.byref(t))
    return st, m.value, t.value


def test_noalloc_mass_matches_lbm_mass_on_consecutive_calls(L):
    p1, phi1, ux1, uy1 = W.small_case(1500, 1400, seed=22)
    p2, phi2 = W.droplet64()
    p3, phi3, ux3, uy3 = W.small_case(70, 45, seed=21, walls=True, gravity=1e-5, u_wall=0.01)
    p4, phi4 = W.precision(n=512, n_drops=8)
    cases = [(p1, phi1, ux1, uy1, "f32", 30), (p2, phi2, None, None, "f64", 40),
             (p3, phi3, ux3, uy3, "f16s", 25), (p4, phi4, None, None, "bf16s", 20)]
    for p, phi, ux, uy, dtype, steps in cases:
        sim = L.Sim(p, dtype)
        sim.init_phi(phi, ux, uy)
        sim.step(steps)
        level, _ = sim.get_state()
        ref_m, ref_t = sim.mass()
        st, m, t = _noalloc(L, p, dtype, level.data_ptr(), sim.stream.cuda_stream)
        assert st == 0, L.load().lbm_create_error()
        assert abs(m - ref_m) <= 1e-12 * abs(ref_m), (dtype, m, ref_m)
        assert abs(t - ref_t) <= 1e-12 * np.abs(phi).sum(), (dtype, t, ref_t)
        sim.close()


def test_noalloc_rejects_grids_beyond_its_limit(L):
    import torch
    p, _ = W.droplet64()
    p = dict(p, nx=20000, ny=20000)          # 4e8 cells > 2^28
    dummy = torch.empty(256, dtype=torch.uint8, device="cuda")
    st, _, _ = _noalloc(L, p, "f32", dummy.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == -6
    assert b"2^28" in L.load().lbm_create_error()
    st, _, _ = _noalloc(L, dict(p, nx=64, ny=64, tau_f=0.4), "f32", dummy.data_ptr(), 0)
    assert st == -1
