"""FP64 CPU oracle of the quasi-incompressible phase-field LBE (arXiv 1507.03521).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, literal statement of
one time step of the scheme of Sec. 3 (Eqs. 22-33), written in C (``orc.c``)
and loaded through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never calls it.

Every function of ``orc.c`` is pinned by ``tests/test_oracle_*.py`` against
facts the paper and the mathematics fix (moment identities of the appendix,
stencil Fourier symbols, conservation, fixed points, the tanh profile of
Eq. 6, the Laplace law of Table I, the linear decay rate of Eq. 19).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_SRC3 = os.path.join(_HERE, "orc3.c")  # the D3Q19 statement, same library
_LIB = os.path.join(_HERE, "liborc.so")

PERIODIC = 0
WALL = 1


def build(force: bool = False) -> str:
    """Compile ``orc.c`` into ``liborc.so`` (plain gcc, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-fPIC", "-shared", _SRC, _SRC3, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liborc_omp.so")


def build_omp(force: bool = False) -> str:
    """The same source built with OpenMP (``liborc_omp.so``): the passes
    over cells run on all host cores, bit-identical to ``liborc.so``."""
    if (not force and os.path.exists(_LIB_OMP)
            and os.path.getmtime(_LIB_OMP) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))):
        return _LIB_OMP
    tmp = _LIB_OMP + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fopenmp",
           "-fPIC", "-shared", _SRC, _SRC3, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def set_threads(n: int, lib: str | None = None) -> int:
    """Threads of the OpenMP build's passes (n <= 0: keep); returns the count."""
    return int(_load(lib).orc_set_threads(int(n)))


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("rho_A", ctypes.c_double), ("rho_B", ctypes.c_double),
        ("phi_A", ctypes.c_double), ("phi_B", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double), ("M", ctypes.c_double),
        ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("gravity", ctypes.c_double), ("rho_ref", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("u_wall_bottom", ctypes.c_double), ("u_wall_top", ctypes.c_double),
    ]


_libs = {}
_dp = ctypes.POINTER(ctypes.c_double)


def build_mutant(k: int, outdir: str) -> str:
    """Build the oracle with mistake number k planted (mutation tests only)."""
    out = os.path.join(outdir, f"liborc_mutant{k}.so")
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
           "-shared", f"-DORC_MUTANT={k}", _SRC, _SRC3, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _load(path: str | None = None):
    if path is None:
        build()
        path = _LIB
    if path in _libs:
        return _libs[path]
    lib = ctypes.CDLL(path)
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [ctypes.POINTER(_Params)]
    lib.orc_params_check.restype = ctypes.c_int
    lib.orc_params_check.argtypes = [ctypes.POINTER(_Params)]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_constants.argtypes = [ctypes.c_void_p, _dp]
    lib.orc_init_phi.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.orc_fields.argtypes = [ctypes.c_void_p] + [_dp] * 6
    lib.orc_mass.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.orc_total_pressure.argtypes = [ctypes.c_void_p, _dp]
    lib.orc_laplace.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, _dp, _dp]
    lib.orc_get_pops.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.orc_set_pops.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.orc_step_count.restype = ctypes.c_long
    lib.orc_step_count.argtypes = [ctypes.c_void_p]
    lib.orc_cell_terms.argtypes = [ctypes.c_double] * 16 + [_dp] * 4
    lib.orc_stencils.argtypes = [ctypes.c_int] * 4 + [_dp] * 4
    lib.orc_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]
    lib.orc_set_gradp_lag.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.orc_step_jitter.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_ulonglong]
    lib.orc3_create.restype = ctypes.c_void_p
    lib.orc3_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int]
    lib.orc3_destroy.argtypes = [ctypes.c_void_p]
    lib.orc3_init_phi.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
    lib.orc3_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.orc3_fields.argtypes = [ctypes.c_void_p] + [_dp] * 7
    lib.orc3_mass.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.orc3_laplace.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 4 + [_dp, _dp]
    lib.orc3_get_pops.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.orc3_step_count.restype = ctypes.c_long
    lib.orc3_step_count.argtypes = [ctypes.c_void_p]
    lib.orc3_stencils.argtypes = [ctypes.c_int] * 3 + [_dp] * 5
    lib.orc3_lattice.argtypes = [ctypes.POINTER(ctypes.c_int)] * 3 + [_dp]
    lib.orc_set_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    _libs[path] = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


@dataclass
class Params:
    """Physical and lattice parameters of one domain (paper notation)."""
    nx: int
    ny: int
    rho_A: float = 1.0
    rho_B: float = 0.1
    phi_A: float = 1.0
    phi_B: float = -1.0
    sigma: float = 0.01
    W: float = 4.0
    M: float = 0.1
    tau_f: float = 0.8
    tau_g: float = 0.8
    gravity: float = 0.0
    rho_ref: float = 1.0
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    u_wall_bottom: float = 0.0
    u_wall_top: float = 0.0

    def _c(self) -> _Params:
        return _Params(self.nx, self.ny, self.rho_A, self.rho_B, self.phi_A, self.phi_B,
                       self.sigma, self.W, self.M, self.tau_f, self.tau_g, self.gravity,
                       self.rho_ref, self.bc_x, self.bc_y, self.u_wall_bottom, self.u_wall_top)


def params_from_dict(d: dict) -> Params:
    keys = Params.__dataclass_fields__.keys()
    return Params(**{k: v for k, v in d.items() if k in keys})


def params_ok(p: Params) -> bool:
    c = p._c()
    return _load().orc_params_check(ctypes.byref(c)) == 0


class Oracle:
    """One FP64 domain stepped by the literal multi-pass scheme."""

    def __init__(self, p: Params | dict, lib: str | None = None, gradp_lag: bool = False):
        if isinstance(p, dict):
            gradp_lag = bool(p.get("gradp_lag", gradp_lag))
            p = params_from_dict(p)
        self.p = p
        self._lib = _load(lib)
        self._cp = p._c()
        h = self._lib.orc_create(ctypes.byref(self._cp))
        if not h:
            raise ValueError(f"oracle rejected parameters {p}")
        self._h = ctypes.c_void_p(h)
        self._lib.orc_set_gradp_lag(self._h, int(gradp_lag))
        self.shape = (p.ny, p.nx)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def constants(self) -> dict:
        out = np.zeros(7)
        self._lib.orc_constants(self._h, _ptr(out))
        return dict(zip(["kappa", "beta", "lambda", "alpha", "gamma", "drho", "nu"], out))

    def init_phi(self, phi0, ux0=None, uy0=None):
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(self.shape)
        ux0 = None if ux0 is None else np.ascontiguousarray(ux0, dtype=np.float64).reshape(self.shape)
        uy0 = None if uy0 is None else np.ascontiguousarray(uy0, dtype=np.float64).reshape(self.shape)
        self._lib.orc_init_phi(self._h, _ptr(phi0), _ptr(ux0), _ptr(uy0))

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    def step_jitter(self, n: int, seed: int = 1):
        """n steps, each after a random +-1 ulp change of every population
        (a conditioning probe for the tests, not part of the scheme)."""
        self._lib.orc_step_jitter(self._h, int(n), int(seed))

    @property
    def step_count(self) -> int:
        return self._lib.orc_step_count(self._h)

    def fields(self) -> dict:
        out = {k: np.zeros(self.shape) for k in ("phi", "rho", "p", "ux", "uy", "mu")}
        self._lib.orc_fields(self._h, *[_ptr(out[k]) for k in ("phi", "rho", "p", "ux", "uy", "mu")])
        return out

    def mass(self):
        m, t = ctypes.c_double(), ctypes.c_double()
        self._lib.orc_mass(self._h, ctypes.byref(m), ctypes.byref(t))
        return m.value, t.value

    def total_pressure(self):
        P = np.zeros(self.shape)
        self._lib.orc_total_pressure(self._h, _ptr(P))
        return P

    def laplace(self, xc, yc, R):
        dP, Re = ctypes.c_double(), ctypes.c_double()
        self._lib.orc_laplace(self._h, float(xc), float(yc), float(R), ctypes.byref(dP), ctypes.byref(Re))
        return dP.value, Re.value

    def pops(self):
        f = np.zeros((9,) + self.shape)
        g = np.zeros((9,) + self.shape)
        self._lib.orc_get_pops(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_pops(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((9,) + self.shape)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((9,) + self.shape)
        self._lib.orc_set_pops(self._h, _ptr(f), _ptr(g))


def cell_terms(alpha, gamma, lam, phi, mu, p, rho, ux, uy, Fx, Fy, grhx, grhy, lmu, gpx, gpy,
               lib=None):
    """f^eq, g^eq, F_i, G_i of one cell (Eqs. 24-29), each a length-9 array."""
    lib = _load(lib)
    out = [np.zeros(9) for _ in range(4)]
    lib.orc_cell_terms(alpha, gamma, lam, phi, mu, p, rho, ux, uy, Fx, Fy, grhx, grhy, lmu,
                       gpx, gpy, *[_ptr(o) for o in out])
    return tuple(out)


def stencils(chi, bc_y=PERIODIC, extrap=False, lib=None):
    """Isotropic gradient and Laplacian of a [ny, nx] field (end of Sec. 3)."""
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    ny, nx = chi.shape
    gx, gy, lap = np.zeros_like(chi), np.zeros_like(chi), np.zeros_like(chi)
    _load(lib).orc_stencils(nx, ny, bc_y, int(extrap), _ptr(chi), _ptr(gx), _ptr(gy), _ptr(lap))
    return gx, gy, lap


def lattice():
    lib = _load()
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = np.zeros(9)
    lib.orc_lattice(cx, cy, _ptr(w))
    return np.array(list(cx)), np.array(list(cy)), w


class Oracle3:
    """One FP64 periodic domain of the D3Q19 statement (orc3.c); fields are
    [nz, ny, nx] arrays, populations [19, nz, ny, nx]."""

    def __init__(self, p: Params | dict, nz: int, lib: str | None = None):
        if isinstance(p, dict):
            p = params_from_dict(p)
        self.p = p
        self._lib = _load(lib)
        self._cp = p._c()
        h = self._lib.orc3_create(ctypes.byref(self._cp), int(nz))
        if not h:
            raise ValueError(f"oracle rejected parameters {p} nz={nz}")
        self._h = ctypes.c_void_p(h)
        self.shape = (int(nz), p.ny, p.nx)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, a):
        return None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)

    def init_phi(self, phi0, ux0=None, uy0=None, uz0=None):
        arrs = [self._arr(a) for a in (phi0, ux0, uy0, uz0)]
        self._keep = arrs
        self._lib.orc3_init_phi(self._h, *[_ptr(a) for a in arrs])

    def step(self, n: int = 1):
        self._lib.orc3_step(self._h, int(n))

    @property
    def step_count(self) -> int:
        return self._lib.orc3_step_count(self._h)

    def fields(self) -> dict:
        keys = ("phi", "rho", "p", "ux", "uy", "uz", "mu")
        out = {k: np.zeros(self.shape) for k in keys}
        self._lib.orc3_fields(self._h, *[_ptr(out[k]) for k in keys])
        return out

    def mass(self):
        m, t = ctypes.c_double(), ctypes.c_double()
        self._lib.orc3_mass(self._h, ctypes.byref(m), ctypes.byref(t))
        return m.value, t.value

    def laplace(self, xc, yc, zc, R):
        dP, Re = ctypes.c_double(), ctypes.c_double()
        self._lib.orc3_laplace(self._h, float(xc), float(yc), float(zc), float(R), ctypes.byref(dP),
                               ctypes.byref(Re))
        return dP.value, Re.value

    def pops(self):
        f = np.zeros((19,) + self.shape)
        g = np.zeros((19,) + self.shape)
        self._lib.orc3_get_pops(self._h, _ptr(f), _ptr(g))
        return f, g


def stencils3(chi):
    """Isotropic D3Q19 gradient and Laplacian of a periodic [nz, ny, nx] field."""
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    nz, ny, nx = chi.shape
    out = [np.zeros_like(chi) for _ in range(4)]
    _load().orc3_stencils(nx, ny, nz, _ptr(chi), *[_ptr(o) for o in out])
    return out


def lattice3():
    cx, cy, cz = [(ctypes.c_int * 19)() for _ in range(3)]
    w = np.zeros(19)
    _load().orc3_lattice(cx, cy, cz, _ptr(w))
    return np.array(cx[:]), np.array(cy[:]), np.array(cz[:]), w
