"""FP64 CPU oracle of the HGKS step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  The product path in ``paper_2005_08736_gb300`` never
imports it, and the oracle shares no code with that path: it is a plain C++
restatement of the scheme of Cao, Pan & Xu (arXiv:2005.08736), Sec. 2.1 and
Sec. 3, compiled here with g++ and loaded through ctypes.

Every function here is argument marshalling; the arithmetic is in
``hgks_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgks_oracle.cpp")
_DEPS = [_SRC, os.path.join(_HERE, "tangent.h"), os.path.join(_HERE, "counted.h")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhgks_oracle.so")
_TAN_PATH = os.path.join(_OUT_DIR, "libhgks_oracle_tangent.so")
_CNT_PATH = os.path.join(_OUT_DIR, "libhgks_oracle_count.so")
_lock = threading.Lock()
_lib = None
_tan = None
_cnt = None

RECON_LINEAR, RECON_WENO_JS, RECON_WENO_Z = 0, 1, 2
FLUX_SMOOTH, FLUX_FULL = 0, 1


def _compile(path: str, extra, force: bool) -> str:
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= max(os.path.getmtime(f) for f in _DEPS)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    omp = [] if "-DORACLE_COUNT" in extra else ["-fopenmp"]  # the tallies need one thread
    cmd = ["g++", "-std=c++17", "-O2", *omp, "-ffp-contract=off", "-fPIC",
           "-shared", "-Wl,-Bsymbolic", *extra, "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _built(path: str, extra) -> str:
    """Compile one variant if its library is missing or older than the source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    return _compile(path, extra, False)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, OpenMP, no FP contraction): the plain
    FP64 build, the dual-number tangent build and the operation-counting build
    (one thread) of the same source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    _compile(_TAN_PATH, ["-DORACLE_TANGENT"], force)
    _compile(_CNT_PATH, ["-DORACLE_COUNT"], force)
    return _compile(_LIB_PATH, [], force)


class OracleConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("x0", ctypes.c_double), ("lx", ctypes.c_double),
        ("y0", ctypes.c_double), ("ly", ctypes.c_double),
        ("z0", ctypes.c_double), ("lz", ctypes.c_double),
        ("y_stretch", ctypes.c_int), ("stretch_b", ctypes.c_double),
        ("bc_y", ctypes.c_int),
        ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("visc_law", ctypes.c_int),
        ("mu_ref", ctypes.c_double), ("T_ref", ctypes.c_double), ("visc_exp", ctypes.c_double),
        ("T_wall", ctypes.c_double), ("force_x", ctypes.c_double),
        ("recon", ctypes.c_int), ("flux", ctypes.c_int),
        ("tau_num_C", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("force_mode", ctypes.c_int), ("mass_flux", ctypes.c_double),
        ("char_recon", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_built(_LIB_PATH, []))
            d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            pd = ctypes.POINTER(ctypes.c_double)
            L.oracle_create.restype = vp
            L.oracle_create.argtypes = [ctypes.POINTER(OracleConfig)]
            L.oracle_destroy.argtypes = [vp]
            L.oracle_set_state.argtypes = [vp, pd]
            L.oracle_get_state.argtypes = [vp, pd]
            L.oracle_step.restype = d
            L.oracle_step.argtypes = [vp, i, d]
            L.oracle_time.restype = d
            L.oracle_time.argtypes = [vp]
            L.oracle_last_force.restype = d
            L.oracle_last_force.argtypes = [vp]
            L.oracle_threads.restype = i
            L.oracle_threads.argtypes = []
            L.oracle_cfl_dt.restype = d
            L.oracle_cfl_dt.argtypes = [vp]
            L.oracle_rhs.argtypes = [vp, d, pd, pd]
            L.oracle_widths.argtypes = [vp, i, pd]
            L.oracle_padded.argtypes = [vp, pd]
            L.oracle_moments.argtypes = [d, d, d, d, d, pd, pd, pd, pd, pd, pd]
            L.oracle_slope.argtypes = [pd, d, pd, pd]
            L.oracle_kinetic.argtypes = [pd, pd, d, pd, pd]
            L.oracle_compat.argtypes = [pd, pd, d, pd]
            L.oracle_time_integrals.argtypes = [d, d, pd]
            L.oracle_s2o4_stage1.restype = d
            L.oracle_s2o4_stage1.argtypes = [d, d, d, d]
            L.oracle_s2o4_stage2.restype = d
            L.oracle_s2o4_stage2.argtypes = [d, d, d, d, d]
            L.oracle_weno5_right.restype = d
            L.oracle_weno5_right.argtypes = [pd, i]
            L.oracle_weno5_left.restype = d
            L.oracle_weno5_left.argtypes = [pd, i]
            L.oracle_tangential.argtypes = [pd, i, pd, pd]
            L.oracle_flux_point.argtypes = [ctypes.POINTER(OracleConfig), pd, d, pd, pd]
            L.oracle_char_basis.argtypes = [pd, d, pd, pd]
            L.oracle_normal_end_values.argtypes = [pd, i, i, d, pd]
            L.oracle_tangential_vec.argtypes = [pd, i, i, pd, d, pd, pd]
            _lib = L
    return _lib


def tangent_lib():
    """The tangent build: the same solver API plus oracle_set/get_tangent."""
    global _tan
    with _lock:
        if _tan is None:
            L = ctypes.CDLL(_built(_TAN_PATH, ["-DORACLE_TANGENT"]))
            d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            pd = ctypes.POINTER(ctypes.c_double)
            L.oracle_create.restype = vp
            L.oracle_create.argtypes = [ctypes.POINTER(OracleConfig)]
            L.oracle_destroy.argtypes = [vp]
            for name in ("oracle_set_state", "oracle_get_state", "oracle_set_tangent",
                         "oracle_get_tangent"):
                getattr(L, name).argtypes = [vp, pd]
            L.oracle_step.restype = d
            L.oracle_step.argtypes = [vp, i, d]
            _tan = L
    return _tan


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Config:
    """Problem statement of the scheme (oracle side): grid, gas, viscosity, modes."""
    nx: int
    ny: int
    nz: int
    lx: float = 2 * np.pi
    ly: float = 2 * np.pi
    lz: float = 2 * np.pi
    x0: float = 0.0
    y0: float = 0.0
    z0: float = 0.0
    y_stretch: int = 0
    stretch_b: float = 2.0
    bc_y: int = 0
    gamma: float = 1.4
    prandtl: float = 0.72
    visc_law: int = 0
    mu_ref: float = 1.0 / 1600.0
    T_ref: float = 1.0
    visc_exp: float = 0.76
    T_wall: float = 1.0
    force_x: float = 0.0
    recon: int = RECON_LINEAR
    flux: int = FLUX_SMOOTH
    tau_num_C: float = 0.0
    cfl: float = 0.5
    force_mode: int = 0
    mass_flux: float = 0.0
    char_recon: int = 0

    def c_struct(self) -> OracleConfig:
        return OracleConfig(**{k: getattr(self, k) for k, _ in OracleConfig._fields_})


class Solver:
    """The oracle's HGKS solver: conservative cell averages [5][nz][ny][nx], FP64."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self._c = cfg.c_struct()
        self._h = lib().oracle_create(ctypes.byref(self._c))
        self.shape = (5, cfg.nz, cfg.ny, cfg.nx)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_destroy(h)
            self._h = None

    def set_state(self, cons) -> None:
        a = _f64(cons)
        assert a.shape == self.shape
        lib().oracle_set_state(self._h, _p(a))

    def state(self) -> np.ndarray:
        out = np.empty(self.shape)
        lib().oracle_get_state(self._h, _p(out))
        return out

    def step(self, nsteps: int = 1, dt: float = 0.0) -> float:
        return lib().oracle_step(self._h, int(nsteps), float(dt))

    @property
    def t(self) -> float:
        return lib().oracle_time(self._h)

    def cfl_dt(self) -> float:
        return lib().oracle_cfl_dt(self._h)

    @property
    def last_force(self) -> float:
        """Streamwise force f_x of the last step (Sec. 3.3)."""
        return lib().oracle_last_force(self._h)

    def rhs(self, dt: float):
        L = np.empty(self.shape)
        dL = np.empty(self.shape)
        lib().oracle_rhs(self._h, float(dt), _p(L), _p(dL))
        return L, dL

    def widths(self, d: int) -> np.ndarray:
        n = (self.cfg.nx, self.cfg.ny, self.cfg.nz)[d]
        out = np.empty(n)
        lib().oracle_widths(self._h, d, _p(out))
        return out

    def padded(self) -> np.ndarray:
        c = self.cfg
        out = np.empty((5, c.nz + 6, c.ny + 6, c.nx + 6))
        lib().oracle_padded(self._h, _p(out))
        return out


def count_lib():
    """The counting build: the solver API plus oracle_count_get / _reset."""
    global _cnt
    with _lock:
        if _cnt is None:
            L = ctypes.CDLL(_built(_CNT_PATH, ["-DORACLE_COUNT"]))
            d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            pd = ctypes.POINTER(ctypes.c_double)
            L.oracle_create.restype = vp
            L.oracle_create.argtypes = [ctypes.POINTER(OracleConfig)]
            L.oracle_destroy.argtypes = [vp]
            L.oracle_set_state.argtypes = [vp, pd]
            L.oracle_get_state.argtypes = [vp, pd]
            L.oracle_step.restype = d
            L.oracle_step.argtypes = [vp, i, d]
            L.oracle_count_get.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
            L.oracle_count_reset.argtypes = []
            _cnt = L
    return _cnt


COUNT_KEYS = ("add", "mul", "div", "sqrt", "exp", "erfc", "pow")


def threads() -> int:
    """Threads the plain oracle's parallel loops use (OMP_NUM_THREADS, else
    the cores OpenMP sees)."""
    return int(lib().oracle_threads())


def count_step(cfg: Config, cons, nsteps: int = 1, dt: float = 0.0):
    """Run the counting build for nsteps from the conservative state cons:
    returns (final state, tallies of the oracle's operations over the run,
    a dict over COUNT_KEYS).  Single-threaded."""
    L = count_lib()
    c = cfg.c_struct()
    h = L.oracle_create(ctypes.byref(c))
    try:
        a = _f64(cons)
        L.oracle_set_state(h, _p(a))
        L.oracle_count_reset()
        L.oracle_step(h, int(nsteps), float(dt))
        out = (ctypes.c_ulonglong * 7)()
        L.oracle_count_get(out)
        state = np.empty((5, cfg.nz, cfg.ny, cfg.nx))
        L.oracle_get_state(h, _p(state))
    finally:
        L.oracle_destroy(h)
    return state, dict(zip(COUNT_KEYS, (int(x) for x in out)))


class TangentSolver:
    """Dual-number tangent run of the oracle: the same step computed with
    forward-mode dual numbers, so that along with Q^n it carries
    dQ^n = (dQ^n/dQ^0) dQ^0 for one direction dQ^0.  dt is held fixed (a
    positive dt is required: the CFL step would make dt depend on the state)."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self._c = cfg.c_struct()
        self._h = tangent_lib().oracle_create(ctypes.byref(self._c))
        self.shape = (5, cfg.nz, cfg.ny, cfg.nx)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            tangent_lib().oracle_destroy(h)
            self._h = None

    def set_state(self, cons, dcons) -> None:
        a, da = _f64(cons), _f64(dcons)
        assert a.shape == self.shape and da.shape == self.shape
        tangent_lib().oracle_set_state(self._h, _p(a))
        tangent_lib().oracle_set_tangent(self._h, _p(da))

    def state(self) -> np.ndarray:
        out = np.empty(self.shape)
        tangent_lib().oracle_get_state(self._h, _p(out))
        return out

    def tangent(self) -> np.ndarray:
        out = np.empty(self.shape)
        tangent_lib().oracle_get_tangent(self._h, _p(out))
        return out

    def step(self, nsteps: int, dt: float) -> float:
        if not dt > 0.0:
            raise ValueError("the tangent run needs a fixed dt > 0")
        return tangent_lib().oracle_step(self._h, int(nsteps), float(dt))


# ---- single pieces -------------------------------------------------------------

def moments(U, V, W, lam, K):
    out = [np.empty(10) for _ in range(5)] + [np.empty(4)]
    lib().oracle_moments(float(U), float(V), float(W), float(lam), float(K), *[_p(o) for o in out])
    return dict(uf=out[0], up=out[1], un=out[2], v=out[3], w=out[4], xi=out[5])


def slope(Q, gamma, b):
    a = np.empty(5)
    lib().oracle_slope(_p(_f64(Q)), float(gamma), _p(_f64(b)), _p(a))
    return a


def kinetic(Q, dQ, gamma):
    a = np.empty((3, 5))
    A = np.empty(5)
    lib().oracle_kinetic(_p(_f64(Q)), _p(_f64(dQ)), float(gamma), _p(a), _p(A))
    return a, A


def compat(Ql, Qr, gamma):
    out = np.empty(5)
    lib().oracle_compat(_p(_f64(Ql)), _p(_f64(Qr)), float(gamma), _p(out))
    return out


def time_integrals(T, tau):
    q = np.empty(6)
    lib().oracle_time_integrals(float(T), float(tau), _p(q))
    return q


def s2o4_stage1(Qn, L0, dL0, dt):
    return lib().oracle_s2o4_stage1(float(Qn), float(L0), float(dL0), float(dt))


def s2o4_stage2(Qn, L0, dL0, dL1, dt):
    return lib().oracle_s2o4_stage2(float(Qn), float(L0), float(dL0), float(dL1), float(dt))


def weno5_right(q, mode):
    return lib().oracle_weno5_right(_p(_f64(q)), int(mode))


def weno5_left(q, mode):
    return lib().oracle_weno5_left(_p(_f64(q)), int(mode))


def tangential(f, mode):
    val = np.empty(2)
    der = np.empty(2)
    lib().oracle_tangential(_p(_f64(f)), int(mode), _p(val), _p(der))
    return val, der


def flux_point(cfg: Config, st, dt):
    """st: [3][4][5] = states (l, r, 0) x (value, d/dn, d/dt1, d/dt2) x vars, local frame."""
    c = cfg.c_struct()
    F = np.empty(5)
    dF = np.empty(5)
    lib().oracle_flux_point(ctypes.byref(c), _p(_f64(st)), float(dt), _p(F), _p(dF))
    return F, dF


def char_basis(Qm, gamma):
    """Right eigenvectors R (columns) of the local-frame Euler Jacobian at Qm and R^{-1}."""
    R, L = np.empty((5, 5)), np.empty((5, 5))
    lib().oracle_char_basis(_p(_f64(Qm)), float(gamma), _p(R), _p(L))
    return R, L


def normal_end_values(qc, mode, use_char, gamma=1.4):
    """WENO5 end values [4][5] of the two cells beside a face from qc[6][5]."""
    out = np.empty((4, 5))
    lib().oracle_normal_end_values(_p(_f64(qc)), int(mode), int(use_char), float(gamma), _p(out))
    return out


def tangential_vec(f, mode, use_char, Qm, gamma=1.4):
    """Values and derivatives [2][5] at the Gauss abscissae from face averages f[5][5]."""
    val, der = np.empty((2, 5)), np.empty((2, 5))
    lib().oracle_tangential_vec(_p(_f64(f)), int(mode), int(use_char), _p(_f64(Qm)), float(gamma),
                                _p(val), _p(der))
    return val, der


def conservative(prim, gamma):
    """Conservative variables from primitive (rho, u, v, w, p) [5, ...] (oracle side)."""
    prim = np.asarray(prim, dtype=np.float64)
    rho, u, v, w, p = prim
    return np.stack([rho, rho * u, rho * v, rho * w,
                     p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])
