"""Host-side tests of the C ABI (no GPU): the library builds for sm_103a,
loads, exports exactly the entry points include/lbm.h declares, matches the
header's struct layout, and validates parameters without touching CUDA."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1507_03521_gb300 import build, lbm
    build.build()
    return lbm.load()


def _declared():
    txt = open(HEADER).read()
    return set(re.findall(r"LBM_API[^;(]*?\b(lbm3?_\w+)\s*\(", txt))


def test_exports_match_header(lib):
    from paper_1507_03521_gb300 import lbm
    declared = _declared()
    assert declared == set(lbm.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == declared
    for name in declared:
        assert hasattr(lib, name)


def test_debug_build_exports_the_same_entry_points():
    """liblbm_debug.so (LBM_DEBUG: bounds-checked indices) builds from the
    same sources and exports exactly the same entry points."""
    from paper_1507_03521_gb300 import build, lbm
    path = build.build(debug=True)
    assert path == lbm.LIB_DEBUG_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    assert {l.split()[-1] for l in out.splitlines() if " T " in l} == _declared()
    dl = lbm.load_debug()
    assert dl is not lbm.load() and dl.lbm_version() == 1


def test_params_layout_matches_header(tmp_path):
    from paper_1507_03521_gb300 import lbm
    src = tmp_path / "off.c"
    names = [f[0] for f in lbm.CParams._fields_]
    body = "\n".join(f'printf("%zu\\n", offsetof(lbm_params, {n}));' for n in names)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\nint main(void){\n'
                   + body + '\nprintf("%zu\\n", sizeof(lbm_params));\nreturn 0;}\n')
    exe = tmp_path / "off"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals[:-1] == [getattr(lbm.CParams, n).offset for n in names]
    assert vals[-1] == ctypes.sizeof(lbm.CParams)


def _params(**kw):
    from paper_1507_03521_gb300 import workloads
    p, _ = workloads.droplet64()
    p.update(kw)
    return p


def test_version_and_sizes(lib):
    from paper_1507_03521_gb300 import lbm
    assert lib.lbm_version() == 1
    sb32, wb32 = lbm.buffer_sizes(_params(), "f32")
    sb64, wb64 = lbm.buffer_sizes(_params(), "f64")
    sb16, _ = lbm.buffer_sizes(_params(), "f16s")
    sb16d, _ = lbm.buffer_sizes(_params(), "f16d")
    N = 64 * 64
    assert sb32 == 2 * 18 * 4 * N and sb64 == 2 * 18 * 8 * N
    assert sb16d == 2 * (4 + 19 * 2) * N  # 17 deviations and the two reference words
    assert sb16 == 2 * (4 + 17 * 2) * N
    assert sb32 % 256 == 0 and wb32 % 256 == 0 and wb64 > wb32


@pytest.mark.parametrize("bad", [dict(tau_f=0.5), dict(tau_g=0.2), dict(rho_B=0.0), dict(W=-1.0),
                                 dict(nx=4), dict(phi_A=-1.0), dict(bc_x=1), dict(bc_y=3),
                                 dict(sigma=float("nan"))])
def test_create_rejects_bad_params(lib, bad):
    from paper_1507_03521_gb300 import lbm
    cp = lbm.make_params(_params(**bad), "f32")
    h = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(cp), None, ctypes.byref(h)) == -1
    assert not h.value
    assert len(lib.lbm_create_error()) > 0
    cp = lbm.make_params(_params(), "f32")
    cp.dtype = 9
    assert lib.lbm_create(ctypes.byref(cp), None, ctypes.byref(h)) == -1


def test_handle_state_machine_without_gpu(lib):
    """Create/bind/step order checks are host logic: no CUDA call is made
    before buffers are bound and the state initialised."""
    from paper_1507_03521_gb300 import lbm
    cp = lbm.make_params(_params(), "f32")
    h = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(cp), None, ctypes.byref(h)) == 0
    assert lib.lbm_step(h, 1) == -5                      # buffers not bound
    assert b"not bound" in lib.lbm_last_error(h)
    sb, wb = lbm.buffer_sizes(_params(), "f32")
    assert lib.lbm_bind_buffers(h, 256, sb - 256, 512, wb) == -6   # too small
    assert lib.lbm_bind_buffers(h, 300, sb, 512, wb) == -1         # misaligned
    assert lib.lbm_bind_buffers(h, 256, sb, 512, wb) == 0          # pointers are not touched
    assert lib.lbm_step(h, 1) == -5                      # not initialised
    assert lib.lbm_step_count(h) == 0
    lib.lbm_destroy(h)


def test_alu_peak_rejects_bad_arguments_without_gpu(lib):
    """Argument checks come before any CUDA call."""
    out = ctypes.c_double()
    assert lib.lbm_alu_peak(3, ctypes.byref(out)) == -1
    assert lib.lbm_alu_peak(-1, ctypes.byref(out)) == -1
    assert lib.lbm_alu_peak(0, None) == -1
