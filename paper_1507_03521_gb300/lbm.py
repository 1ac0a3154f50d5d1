"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``liblbm.so``.  PyTorch provides the device memory (two caller-
owned buffers) and the stream.  There is no CPU fallback: loading fails
loudly when the library is missing or no GPU is present.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

F64, F32, F16S, BF16S, F16D, BF16D = 0, 1, 2, 3, 4, 5
PERIODIC, WALL = 0, 1
DTYPES = {"f64": F64, "f32": F32, "f16s": F16S, "bf16s": BF16S, "f16d": F16D, "bf16d": BF16D}

STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_NONFINITE",
          -4: "LBM_ERR_TIMEOUT", -5: "LBM_ERR_STATE", -6: "LBM_ERR_NOMEM"}

# Every entry point declared in include/lbm.h.
EXPORTS = ["lbm_version", "lbm_buffer_sizes", "lbm_create", "lbm_bind_buffers", "lbm_init_phi",
           "lbm_step", "lbm_fields", "lbm_mass", "lbm_laplace", "lbm_state_bytes",
           "lbm_get_state", "lbm_set_state", "lbm_step_count", "lbm_last_error",
           "lbm_create_error", "lbm_destroy", "lbm_test_unfinished_tiles", "lbm_mass_noalloc",
           "lbm_alu_peak",
           "lbm_batch_buffer_sizes", "lbm_batch_create", "lbm_batch_bind_buffers",
           "lbm_batch_init_phi", "lbm_batch_step", "lbm_batch_set_graph", "lbm_batch_set_segment",
           "lbm_batch_autotune", "lbm_batch_fields", "lbm_batch_mass", "lbm_batch_cells",
           "lbm_batch_step_count", "lbm_batch_segment", "lbm_batch_work_items", "lbm_batch_last_error",
           "lbm_batch_destroy", "lbm_adj_work_bytes", "lbm_adj_reset", "lbm_adj_seed",
           "lbm_adj_step", "lbm_adj_init", "lbm_adj_grads", "lbm_adj_segment", "lbm_adj_set_graph",
           "lbm_adj_recompute", "lbm_adj_reverse_overlap",
           "lbm_slabs_buffer_sizes", "lbm_slabs_create", "lbm_slabs_bind_buffers",
           "lbm_slabs_scatter", "lbm_slabs_gather", "lbm_slabs_step", "lbm_slabs_rows",
           "lbm_slabs_step_count", "lbm_slabs_last_error", "lbm_slabs_destroy",
           "lbm3_buffer_sizes", "lbm3_create", "lbm3_bind_buffers", "lbm3_init_phi", "lbm3_step",
           "lbm3_fields", "lbm3_mass", "lbm3_laplace", "lbm3_step_count", "lbm3_last_error",
           "lbm3_destroy"]


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CParams(ctypes.Structure):
    """Mirror of lbm_params (include/lbm.h)."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("rho_A", ctypes.c_double), ("rho_B", ctypes.c_double),
        ("phi_A", ctypes.c_double), ("phi_B", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double), ("M", ctypes.c_double),
        ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("gravity", ctypes.c_double), ("rho_ref", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("u_wall_bottom", ctypes.c_double), ("u_wall_top", ctypes.c_double),
        ("dtype", ctypes.c_int),
        ("gradp_lag", ctypes.c_int),
    ]


_lib = None
_lib_debug = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
LIB_DEBUG_PATH = os.path.join(HERE, "liblbm_debug.so")


def load(path: str = LIB_PATH):
    """Load liblbm.so (no build, no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = _open(path)
    return _lib


def load_debug():
    """Load liblbm_debug.so, the LBM_DEBUG build (bounds-checked indices),
    built by build.build(debug=True)."""
    global _lib_debug
    if _lib_debug is None:
        _lib_debug = _open(LIB_DEBUG_PATH)
    return _lib_debug


def _open(path: str):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    S = ctypes.c_int
    lib.lbm_version.restype = ctypes.c_int
    lib.lbm_buffer_sizes.restype = S
    lib.lbm_buffer_sizes.argtypes = [ctypes.POINTER(CParams), ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]
    lib.lbm_create.restype = S
    lib.lbm_create.argtypes = [ctypes.POINTER(CParams), _vp, ctypes.POINTER(_vp)]
    lib.lbm_bind_buffers.restype = S
    lib.lbm_bind_buffers.argtypes = [_vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t]
    lib.lbm_init_phi.restype = S
    lib.lbm_init_phi.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int]
    lib.lbm_step.restype = S
    lib.lbm_step.argtypes = [_vp, ctypes.c_int64]
    lib.lbm_fields.restype = S
    lib.lbm_fields.argtypes = [_vp] + [_vp] * 6 + [ctypes.c_int]
    lib.lbm_mass.restype = S
    lib.lbm_mass.argtypes = [_vp, _dp, _dp]
    lib.lbm_laplace.restype = S
    lib.lbm_laplace.argtypes = [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
    lib.lbm_state_bytes.restype = ctypes.c_size_t
    lib.lbm_state_bytes.argtypes = [_vp]
    lib.lbm_get_state.restype = S
    lib.lbm_get_state.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    lib.lbm_set_state.restype = S
    lib.lbm_set_state.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int64]
    lib.lbm_step_count.restype = ctypes.c_int64
    lib.lbm_step_count.argtypes = [_vp]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_last_error.argtypes = [_vp]
    lib.lbm_create_error.restype = ctypes.c_char_p
    lib.lbm_destroy.restype = None
    lib.lbm_destroy.argtypes = [_vp]
    lib.lbm_mass_noalloc.restype = S
    lib.lbm_mass_noalloc.argtypes = [ctypes.POINTER(CParams), _vp, _vp, _dp, _dp]
    lib.lbm_alu_peak.restype = S
    lib.lbm_alu_peak.argtypes = [ctypes.c_int, _dp]
    P = ctypes.POINTER(CParams)
    lib.lbm_batch_buffer_sizes.restype = S
    lib.lbm_batch_buffer_sizes.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t),
                                           ctypes.POINTER(ctypes.c_size_t)]
    lib.lbm_batch_create.restype = S
    lib.lbm_batch_create.argtypes = [P, ctypes.c_int, _vp, ctypes.POINTER(_vp)]
    lib.lbm_batch_bind_buffers.restype = S
    lib.lbm_batch_bind_buffers.argtypes = [_vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t]
    lib.lbm_batch_init_phi.restype = S
    lib.lbm_batch_init_phi.argtypes = [_vp, _vp, ctypes.c_int]
    lib.lbm_batch_step.restype = S
    lib.lbm_batch_step.argtypes = [_vp, ctypes.c_int64]
    lib.lbm_batch_set_graph.restype = S
    lib.lbm_batch_set_graph.argtypes = [_vp, ctypes.c_int]
    lib.lbm_batch_set_segment.restype = S
    lib.lbm_batch_set_segment.argtypes = [_vp, ctypes.c_int]
    lib.lbm_batch_autotune.restype = S
    lib.lbm_batch_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp]
    lib.lbm_batch_fields.restype = S
    lib.lbm_batch_fields.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]
    lib.lbm_batch_mass.restype = S
    lib.lbm_batch_mass.argtypes = [_vp, _dp, _dp]
    lib.lbm_batch_cells.restype = ctypes.c_int64
    lib.lbm_batch_cells.argtypes = [_vp]
    lib.lbm_batch_step_count.restype = ctypes.c_int64
    lib.lbm_batch_step_count.argtypes = [_vp]
    lib.lbm_batch_segment.restype = ctypes.c_int
    lib.lbm_batch_segment.argtypes = [_vp]
    lib.lbm_batch_work_items.restype = ctypes.c_int
    lib.lbm_batch_work_items.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    lib.lbm_batch_last_error.argtypes = [_vp]
    lib.lbm_batch_destroy.restype = None
    lib.lbm_batch_destroy.argtypes = [_vp]
    IP = ctypes.POINTER(ctypes.c_int)
    lib.lbm_slabs_buffer_sizes.restype = S
    lib.lbm_slabs_buffer_sizes.argtypes = [P, ctypes.c_int, IP, ctypes.POINTER(ctypes.c_size_t),
                                           ctypes.POINTER(ctypes.c_size_t)]
    lib.lbm_slabs_create.restype = S
    lib.lbm_slabs_create.argtypes = [P, ctypes.c_int, IP, _vp, ctypes.POINTER(_vp)]
    lib.lbm_slabs_bind_buffers.restype = S
    lib.lbm_slabs_bind_buffers.argtypes = [_vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t]
    lib.lbm_slabs_scatter.restype = S
    lib.lbm_slabs_scatter.argtypes = [_vp, _vp, ctypes.c_int64]
    lib.lbm_slabs_gather.restype = S
    lib.lbm_slabs_gather.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_int64)]
    lib.lbm_slabs_step.restype = S
    lib.lbm_slabs_step.argtypes = [_vp, ctypes.c_int64]
    lib.lbm_slabs_rows.restype = S
    lib.lbm_slabs_rows.argtypes = [_vp, ctypes.c_int, IP, IP]
    lib.lbm_slabs_step_count.restype = ctypes.c_int64
    lib.lbm_slabs_step_count.argtypes = [_vp]
    lib.lbm_slabs_last_error.restype = ctypes.c_char_p
    lib.lbm_slabs_last_error.argtypes = [_vp]
    lib.lbm_slabs_destroy.restype = None
    lib.lbm_slabs_destroy.argtypes = [_vp]
    lib.lbm3_buffer_sizes.restype = S
    lib.lbm3_buffer_sizes.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t),
                                      ctypes.POINTER(ctypes.c_size_t)]
    lib.lbm3_create.restype = S
    lib.lbm3_create.argtypes = [P, ctypes.c_int, _vp, ctypes.POINTER(_vp)]
    lib.lbm3_bind_buffers.restype = S
    lib.lbm3_bind_buffers.argtypes = [_vp, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t]
    lib.lbm3_init_phi.restype = S
    lib.lbm3_init_phi.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.lbm3_step.restype = S
    lib.lbm3_step.argtypes = [_vp, ctypes.c_int64]
    lib.lbm3_fields.restype = S
    lib.lbm3_fields.argtypes = [_vp] + [_vp] * 7
    lib.lbm3_mass.restype = S
    lib.lbm3_mass.argtypes = [_vp, _dp, _dp]
    lib.lbm3_laplace.restype = S
    lib.lbm3_laplace.argtypes = [_vp] + [ctypes.c_double] * 4 + [_dp, _dp]
    lib.lbm3_step_count.restype = ctypes.c_int64
    lib.lbm3_step_count.argtypes = [_vp]
    lib.lbm3_last_error.restype = ctypes.c_char_p
    lib.lbm3_last_error.argtypes = [_vp]
    lib.lbm3_destroy.restype = None
    lib.lbm3_destroy.argtypes = [_vp]
    lib.lbm_adj_work_bytes.restype = S
    lib.lbm_adj_work_bytes.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.lbm_adj_reset.restype = S
    lib.lbm_adj_reset.argtypes = [_vp, _vp]
    lib.lbm_adj_seed.restype = S
    lib.lbm_adj_seed.argtypes = [_vp, _vp, _vp, _vp, _vp, _dp]
    lib.lbm_adj_step.restype = S
    lib.lbm_adj_step.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.lbm_adj_init.restype = S
    lib.lbm_adj_init.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.lbm_adj_grads.restype = S
    lib.lbm_adj_grads.argtypes = [_vp, _vp, _dp, _dp]
    lib.lbm_adj_segment.restype = S
    lib.lbm_adj_segment.argtypes = [_vp, ctypes.c_int64, _vp, ctypes.c_size_t, _vp, _vp, _vp]
    lib.lbm_adj_set_graph.restype = S
    lib.lbm_adj_set_graph.argtypes = [_vp, ctypes.c_int]
    lib.lbm_adj_recompute.restype = S
    lib.lbm_adj_recompute.argtypes = [_vp, ctypes.c_int64, _vp, ctypes.c_size_t]
    lib.lbm_adj_reverse_overlap.restype = S
    lib.lbm_adj_reverse_overlap.argtypes = [_vp, ctypes.c_int64, _vp, ctypes.c_size_t, _vp, _vp, _vp,
                                            ctypes.c_int64, _vp]
    lib.lbm_test_unfinished_tiles.restype = S
    lib.lbm_test_unfinished_tiles.argtypes = [_vp, ctypes.c_int]
    return lib


def make_params(d: dict, dtype) -> CParams:
    """lbm_params from a parameter dict in the paper's notation."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    keys = [f[0] for f in CParams._fields_ if f[0] not in ("dtype", "gradp_lag")]
    return CParams(*[d[k] for k in keys], dtype, int(d.get("gradp_lag", 0)))


def alu_peak(kind: str) -> float:
    """Measured FMA operations per second of the current GPU: kind "f32"
    (scalar), "f32x2" (packed pairs) or "f64" (lbm_alu_peak)."""
    k = {"f32": 0, "f32x2": 1, "f64": 2}[kind]
    out = ctypes.c_double()
    st = load().lbm_alu_peak(k, ctypes.byref(out))
    if st != 0:
        raise LBMError(st, "lbm_alu_peak failed")
    return out.value


def buffer_sizes(d: dict, dtype):
    lib = load()
    cp = make_params(d, dtype)
    sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
    st = lib.lbm_buffer_sizes(ctypes.byref(cp), ctypes.byref(sb), ctypes.byref(wb))
    if st != 0:
        raise LBMError(st, lib.lbm_create_error().decode())
    return sb.value, wb.value


class Sim:
    """One domain on the current CUDA device.

    ``params`` is a dict in the paper's notation (see workloads.py);
    ``dtype`` one of "f64", "f32", "f16s", "bf16s", "f16d", "bf16d".
    Buffers are torch tensors owned by this object; the stream is torch's
    current stream at construction unless one is given.  ``debug`` runs the
    handle on liblbm_debug.so, the bounds-checked LBM_DEBUG build.
    """

    def __init__(self, params: dict, dtype="f32", stream=None, device=None, debug=False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device; none is available")
        self._lib = load_debug() if debug else load()
        self.params = dict(params)
        self.dtype = dtype if isinstance(dtype, str) else {v: k for k, v in DTYPES.items()}[dtype]
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.field_dtype = torch.float64 if self.dtype == "f64" else torch.float32
        self.shape = (params["ny"], params["nx"])
        self._cp = make_params(params, self.dtype)
        h = _vp()
        st = self._lib.lbm_create(ctypes.byref(self._cp), _vp(self.stream.cuda_stream),
                                  ctypes.byref(h))
        if st != 0:
            raise LBMError(st, self._lib.lbm_create_error().decode())
        self._h = h
        sb, wb = buffer_sizes(params, self.dtype)
        self.state_buf = torch.empty(sb, dtype=torch.uint8, device=self.device)
        self.work_buf = torch.empty(wb, dtype=torch.uint8, device=self.device)
        self._check(self._lib.lbm_bind_buffers(h, self.state_buf.data_ptr(), sb,
                                               self.work_buf.data_ptr(), wb))

    # -- plumbing
    def _check(self, st):
        if st != 0:
            raise LBMError(st, self._lib.lbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API
    def _field_tensor(self, a):
        import torch
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a))
        return a.to(device=self.device, dtype=self.field_dtype).contiguous().reshape(self.shape)

    def init_phi(self, phi, ux=None, uy=None):
        """Equilibrium initial state from phi (and optional u): device path."""
        t = [self._field_tensor(a) for a in (phi, ux, uy)]
        self._keep = t  # inputs must live until the stream consumes them
        ptr = [None if a is None else a.data_ptr() for a in t]
        self._check(self._lib.lbm_init_phi(self._h, ptr[0], ptr[1], ptr[2], 0))

    def init_phi_host(self, phi, ux=None, uy=None):
        """Same from host numpy arrays (copied in by the library)."""
        npdt = np.float64 if self.dtype == "f64" else np.float32
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=npdt).reshape(self.shape)
                for a in (phi, ux, uy)]
        ptr = [None if a is None else a.ctypes.data for a in arrs]
        self._check(self._lib.lbm_init_phi(self._h, ptr[0], ptr[1], ptr[2], 1))

    def step(self, n: int = 1):
        self._check(self._lib.lbm_step(self._h, int(n)))

    @property
    def step_count(self) -> int:
        return self._lib.lbm_step_count(self._h)

    def fields(self, names=("phi", "rho", "p", "ux", "uy", "mu")):
        """Device tensors of the current macroscopic fields."""
        import torch
        order = ("phi", "rho", "p", "ux", "uy", "mu")
        out = {k: torch.empty(self.shape, dtype=self.field_dtype, device=self.device)
               for k in names}
        ptr = [out[k].data_ptr() if k in out else None for k in order]
        self._check(self._lib.lbm_fields(self._h, *ptr, 0))
        return out

    def fields_host(self, names=("phi", "rho", "p", "ux", "uy", "mu"), out=None):
        """Host numpy copies of the current fields (library copies out)."""
        order = ("phi", "rho", "p", "ux", "uy", "mu")
        npdt = np.float64 if self.dtype == "f64" else np.float32
        if out is None:
            out = {k: np.empty(self.shape, dtype=npdt) for k in names}
        ptr = [out[k].ctypes.data if k in out else None for k in order]
        self._check(self._lib.lbm_fields(self._h, *ptr, 1))
        return out

    def mass(self):
        m, t = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbm_mass(self._h, ctypes.byref(m), ctypes.byref(t)))
        return m.value, t.value

    def laplace(self, xc, yc, R):
        dP, Re = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbm_laplace(self._h, float(xc), float(yc), float(R),
                                          ctypes.byref(dP), ctypes.byref(Re)))
        return dP.value, Re.value

    def state_bytes(self) -> int:
        return self._lib.lbm_state_bytes(self._h)

    def get_state(self):
        import torch
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        step = ctypes.c_int64()
        self._check(self._lib.lbm_get_state(self._h, buf.data_ptr(), 0, ctypes.byref(step)))
        return buf, step.value

    def set_state(self, buf, step: int):
        self._check(self._lib.lbm_set_state(self._h, buf.data_ptr(), 0, int(step)))

    # -- adjoint (f64 / f32 handles)
    def adj_work(self):
        import torch
        b = ctypes.c_size_t()
        self._check(self._lib.lbm_adj_work_bytes(self._h, ctypes.byref(b)))
        w = torch.empty(b.value, dtype=torch.uint8, device=self.device)
        self._check(self._lib.lbm_adj_reset(self._h, w.data_ptr()))
        return w

    def adj_seed(self, state, target, lam, work):
        t = self._field_tensor(target)
        self._keep_target = t
        loss = ctypes.c_double()
        self._check(self._lib.lbm_adj_seed(self._h, state.data_ptr(), t.data_ptr(),
                                           lam.data_ptr(), work.data_ptr(), ctypes.byref(loss)))
        return loss.value

    def adj_step(self, state, lam_next, lam, work):
        self._check(self._lib.lbm_adj_step(self._h, state.data_ptr(), lam_next.data_ptr(),
                                           lam.data_ptr(), work.data_ptr()))

    def adj_init(self, phi0, lam0, work):
        import torch
        ph = self._field_tensor(phi0)
        out = torch.empty(self.shape, dtype=self.field_dtype, device=self.device)
        self._check(self._lib.lbm_adj_init(self._h, ph.data_ptr(), lam0.data_ptr(),
                                           out.data_ptr(), work.data_ptr()))
        return out

    def adj_segment(self, n, states, level_stride, lam, lam_tmp, work):
        """n reverse steps of one checkpoint segment (lbm_adj_segment):
        states[0] holds the checkpoint; lam goes from lambda_{t0+n} to
        lambda_{t0}."""
        self._check(self._lib.lbm_adj_segment(self._h, int(n), states.data_ptr(), int(level_stride),
                                              lam.data_ptr(), lam_tmp.data_ptr(), work.data_ptr()))

    def adj_recompute(self, n, states, level_stride):
        """Levels 1 .. n-1 of `states` from level 0 (lbm_adj_recompute)."""
        self._check(self._lib.lbm_adj_recompute(self._h, int(n), states.data_ptr(), int(level_stride)))

    def adj_reverse_overlap(self, n, states, level_stride, lam, lam_tmp, work, n_next=0,
                            next_states=None):
        """n reverse steps of `states` (already recomputed) while a second
        stream recomputes n_next levels of `next_states` from its level 0
        (lbm_adj_reverse_overlap)."""
        nxt = next_states.data_ptr() if next_states is not None else None
        self._check(self._lib.lbm_adj_reverse_overlap(
            self._h, int(n), states.data_ptr(), int(level_stride), lam.data_ptr(), lam_tmp.data_ptr(),
            work.data_ptr(), int(n_next), nxt))

    def test_unfinished_tiles(self, on: bool):
        """Test hook: tile loads that never finish, so their bounded waits
        run out (lbm_test_unfinished_tiles)."""
        self._check(self._lib.lbm_test_unfinished_tiles(self._h, int(bool(on))))

    def adj_set_graph(self, on: bool):
        self._check(self._lib.lbm_adj_set_graph(self._h, int(bool(on))))

    def adj_grads(self, work):
        dM, dS = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbm_adj_grads(self._h, work.data_ptr(), ctypes.byref(dM),
                                            ctypes.byref(dS)))
        return dM.value, dS.value


class Slabs:
    """One domain as y-slabs stepped separately with device-to-device ghost
    exchange (``lbm_slabs_*``).  ``n_slabs`` even slabs, or explicit
    ``row_starts``.  States are whole-domain levels as ``Sim.get_state``
    returns them; the slabs run on ``stream`` (default: torch's current)."""

    def __init__(self, params: dict, dtype="f32", n_slabs=2, row_starts=None, stream=None,
                 device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device; none is available")
        self._lib = load()
        self.params = dict(params)
        self.dtype = dtype
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._cp = make_params(self.params, dtype)
        if row_starts is not None:
            n_slabs = len(row_starts)
            self._starts = (ctypes.c_int * n_slabs)(*[int(r) for r in row_starts])
        else:
            self._starts = None
        self.n = int(n_slabs)
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        st = self._lib.lbm_slabs_buffer_sizes(ctypes.byref(self._cp), self.n, self._starts,
                                              ctypes.byref(sb), ctypes.byref(wb))
        if st != 0:
            raise LBMError(st, self._lib.lbm_create_error().decode())
        h = _vp()
        st = self._lib.lbm_slabs_create(ctypes.byref(self._cp), self.n, self._starts,
                                        _vp(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise LBMError(st, self._lib.lbm_create_error().decode())
        self._h = h
        self.state_buf = torch.empty(sb.value, dtype=torch.uint8, device=self.device)
        self.work_buf = torch.empty(wb.value, dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        self._check(self._lib.lbm_slabs_bind_buffers(h, self.state_buf.data_ptr(), sb.value,
                                                     self.work_buf.data_ptr(), wb.value))

    def _check(self, st):
        if st != 0:
            raise LBMError(st, self._lib.lbm_slabs_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self._lib.lbm_slabs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rows(self):
        out = []
        for i in range(self.n):
            a, b = ctypes.c_int(), ctypes.c_int()
            self._check(self._lib.lbm_slabs_rows(self._h, i, ctypes.byref(a), ctypes.byref(b)))
            out.append((a.value, b.value))
        return out

    @property
    def step_count(self) -> int:
        return self._lib.lbm_slabs_step_count(self._h)

    def scatter(self, level, step: int = 0):
        """Load a whole-domain level (uint8 device tensor)."""
        self._level_keep = level
        self._check(self._lib.lbm_slabs_scatter(self._h, level.data_ptr(), int(step)))

    def gather(self, out=None):
        """The current state as a whole-domain level; returns (tensor, step)."""
        import torch
        if out is None:
            out = torch.zeros_like(self._level_keep)
        step = ctypes.c_int64()
        self._check(self._lib.lbm_slabs_gather(self._h, out.data_ptr(), ctypes.byref(step)))
        return out, step.value

    def step(self, n=1):
        self._check(self._lib.lbm_slabs_step(self._h, int(n)))


class Sim3:
    """One periodic D3Q19 domain (lbm3_*): fields are [nz, ny, nx] tensors of
    the field type; ``dtype`` "f32" or "f64"."""

    def __init__(self, params: dict, nz: int, dtype="f32", stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device; none is available")
        self._lib = load()
        self.params = dict(params)
        self.nz = int(nz)
        self.dtype = dtype
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.field_dtype = torch.float64 if dtype == "f64" else torch.float32
        self.shape = (self.nz, params["ny"], params["nx"])
        self._cp = make_params(self.params, dtype)
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        st = self._lib.lbm3_buffer_sizes(ctypes.byref(self._cp), self.nz, ctypes.byref(sb),
                                         ctypes.byref(wb))
        if st != 0:
            raise LBMError(st, self._lib.lbm_create_error().decode())
        h = _vp()
        st = self._lib.lbm3_create(ctypes.byref(self._cp), self.nz, _vp(self.stream.cuda_stream),
                                   ctypes.byref(h))
        if st != 0:
            raise LBMError(st, self._lib.lbm_create_error().decode())
        self._h = h
        self.state_buf = torch.empty(sb.value, dtype=torch.uint8, device=self.device)
        self.work_buf = torch.empty(wb.value, dtype=torch.uint8, device=self.device)
        self._check(self._lib.lbm3_bind_buffers(h, self.state_buf.data_ptr(), sb.value,
                                                self.work_buf.data_ptr(), wb.value))

    def _check(self, st):
        if st != 0:
            raise LBMError(st, self._lib.lbm3_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self._lib.lbm3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _t(self, a):
        import torch
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a))
        return a.to(device=self.device, dtype=self.field_dtype).contiguous().reshape(self.shape)

    def init_phi(self, phi, ux=None, uy=None, uz=None):
        t = [self._t(a) for a in (phi, ux, uy, uz)]
        self._keep = t
        self._check(self._lib.lbm3_init_phi(self._h, *[None if a is None else a.data_ptr() for a in t]))

    def step(self, n: int = 1):
        self._check(self._lib.lbm3_step(self._h, int(n)))

    @property
    def step_count(self) -> int:
        return self._lib.lbm3_step_count(self._h)

    def fields(self, names=("phi", "rho", "p", "ux", "uy", "uz", "mu")):
        import torch
        out = {k: torch.empty(self.shape, dtype=self.field_dtype, device=self.device) for k in names}
        ptr = [out[k].data_ptr() if k in out else None
               for k in ("phi", "rho", "p", "ux", "uy", "uz", "mu")]
        self._check(self._lib.lbm3_fields(self._h, *ptr))
        self.stream.synchronize()
        return out

    def mass(self):
        m, t = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbm3_mass(self._h, ctypes.byref(m), ctypes.byref(t)))
        return m.value, t.value

    def laplace(self, xc, yc, zc, R):
        dP, Re = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbm3_laplace(self._h, float(xc), float(yc), float(zc), float(R),
                                           ctypes.byref(dP), ctypes.byref(Re)))
        return dP.value, Re.value


class Batch:
    """Many independent domains advanced together (one persistent launch per
    strip width per step).

    ``params_list``: parameter dicts (every nx a multiple of 8); ``dtype``
    shared by all.  Runs on its own torch stream so that CUDA-graph replay
    is possible.  Fields come back as a list of per-domain tensors.
    """

    def __init__(self, params_list, dtype="f32", device=None, graph=False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device; none is available")
        self._lib = load()
        self.dtype = dtype
        self.params = [dict(p) for p in params_list]
        self.n = len(self.params)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = torch.cuda.Stream(self.device)
        self.field_dtype = torch.float64 if dtype == "f64" else torch.float32
        arr = (CParams * self.n)(*[make_params(p, dtype) for p in self.params])
        self._arr = arr
        sb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        st = self._lib.lbm_batch_buffer_sizes(arr, self.n, ctypes.byref(sb), ctypes.byref(wb))
        if st != 0:
            raise LBMError(st, self._lib.lbm_create_error().decode())
        h = _vp()
        st = self._lib.lbm_batch_create(arr, self.n, _vp(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise LBMError(st, self._lib.lbm_create_error().decode())
        self._h = h
        self.state_buf = torch.empty(sb.value, dtype=torch.uint8, device=self.device)
        self.work_buf = torch.empty(wb.value, dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        self._check(self._lib.lbm_batch_bind_buffers(h, self.state_buf.data_ptr(), sb.value,
                                                     self.work_buf.data_ptr(), wb.value))
        if graph:
            self._check(self._lib.lbm_batch_set_graph(h, 1))
        self.shapes = [(p["ny"], p["nx"]) for p in self.params]
        self.offsets = np.concatenate([[0], np.cumsum([a * b for a, b in self.shapes])])

    def _check(self, st):
        if st != 0:
            raise LBMError(st, self._lib.lbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def cells(self) -> int:
        return self._lib.lbm_batch_cells(self._h)

    @property
    def step_count(self) -> int:
        return self._lib.lbm_batch_step_count(self._h)

    @property
    def segment(self) -> int:
        return self._lib.lbm_batch_segment(self._h)

    def work_items(self):
        """(items of the strip kernel, items of the narrow-strip kernel) per step."""
        w, n = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.lbm_batch_work_items(self._h, ctypes.byref(w), ctypes.byref(n)))
        return w.value, n.value

    def init_phi(self, phis):
        import torch
        flat = np.concatenate([np.ascontiguousarray(p, dtype=np.float64).ravel() for p in phis])
        t = torch.from_numpy(flat).to(device=self.device, dtype=self.field_dtype)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._keep = t
        self._check(self._lib.lbm_batch_init_phi(self._h, t.data_ptr(), 0))

    def step(self, n=1):
        self._check(self._lib.lbm_batch_step(self._h, int(n)))

    def set_segment(self, seg_h):
        self._check(self._lib.lbm_batch_set_segment(self._h, int(seg_h)))

    def autotune(self, steps=3):
        seg, ms = ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.lbm_batch_autotune(self._h, int(steps), ctypes.byref(seg),
                                                 ctypes.byref(ms)))
        return seg.value, ms.value

    def fields(self):
        import torch
        out = {k: torch.empty(int(self.offsets[-1]), dtype=self.field_dtype, device=self.device)
               for k in ("phi", "ux", "uy", "p")}
        self._check(self._lib.lbm_batch_fields(self._h, out["phi"].data_ptr(), out["ux"].data_ptr(),
                                               out["uy"].data_ptr(), out["p"].data_ptr(), 0))
        self.stream.synchronize()
        res = []
        for i, (ny, nx) in enumerate(self.shapes):
            a, b = int(self.offsets[i]), int(self.offsets[i + 1])
            res.append({k: v[a:b].reshape(ny, nx) for k, v in out.items()})
        return res

    def mass(self):
        m = np.zeros(self.n)
        t = np.zeros(self.n)
        self._check(self._lib.lbm_batch_mass(self._h, m.ctypes.data_as(_dp), t.ctypes.data_as(_dp)))
        return m, t


@dataclass
class HostRun:
    fields: dict
    mass: tuple


def run_host(params: dict, phi0: np.ndarray, steps: int, dtype="f32", ux0=None, uy0=None,
             names=("phi", "ux", "uy", "p")) -> HostRun:
    """End-to-end call with host buffers: copy phi0 in, step, copy fields out."""
    sim = Sim(params, dtype)
    try:
        sim.init_phi_host(phi0, ux0, uy0)
        sim.step(steps)
        out = sim.fields_host(names)
        return HostRun(out, sim.mass())
    finally:
        sim.close()
