"""lbm_alu_peak: the measured FMA rates that the step's arithmetic is
compared with.  Checks that they are finite, repeat, and order as the
hardware's unit counts do (FP64 far below FP32; packed pairs no slower
than scalar FP32)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1507_03521_gb300 import build, lbm
    build.build()
    return lbm


def test_alu_peaks_are_plausible(L):
    a = {k: L.alu_peak(k) for k in ("f32", "f32x2", "f64")}
    b = {k: L.alu_peak(k) for k in ("f32", "f32x2", "f64")}
    for k in a:
        assert a[k] > 0 and abs(a[k] - b[k]) <= 0.1 * a[k], (k, a[k], b[k])
    assert a["f64"] < a["f32"] / 8
    assert a["f32x2"] >= 0.9 * a["f32"]
