"""ctypes binding of the C ABI in include/hgks.h (argument marshalling only).

Every step of the scheme runs in the CUDA kernels of libhgks.so; this module
only converts Python values to the C structs and pointers of the ABI.  It
raises if the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhgks.so")

HGKS_OK, HGKS_E_INVAL, HGKS_E_NOMEM, HGKS_E_CUDA, HGKS_E_NONPHYSICAL, HGKS_E_TIMEOUT, \
    HGKS_E_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "E_INVAL", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_NONPHYSICAL",
                5: "E_TIMEOUT", 6: "E_UNSUPPORTED"}

# Entry points declared in include/hgks.h.
EXPORTS = ["hgks_default_config", "hgks_create", "hgks_destroy", "hgks_init_state",
           "hgks_init_conservative", "hgks_get_state", "hgks_step", "hgks_diagnostics",
           "hgks_adjoint_step", "hgks_profile_step", "hgks_step_noalloc", "hgks_last_error",
           "hgks_ensemble_create", "hgks_ensemble_step", "hgks_ensemble_destroy",
           "hgks_ensemble_last_error", "hgks_autotune", "hgks_set_sweep_shape",
           "hgks_turbulence_stats", "hgks_measure_fp_peaks", "hgks_channel_stats",
           "hgks_set_time", "hgks_count_flops", "hgks_channel_compose", "hgks_cell_widths",
           "hgks_kinetic_energy", "hgks_history_start", "hgks_history_stop",
           "hgks_history_read", "hgks_ensemble_set_batched"]
KERNEL_CLASSES = ["cfl", "ghost", "face_fields", "flux_stage1", "flux_stage2", "update"]
CHANNEL_PROFILES = ("rho", "rhoU", "U", "V", "W", "UV", "UU", "T", "y", "y_plus", "U_plus",
                    "uv_plus", "dUp_dYp", "total_stress_residual")


class HgksConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("x0", ctypes.c_double), ("lx", ctypes.c_double),
        ("y0", ctypes.c_double), ("ly", ctypes.c_double),
        ("z0", ctypes.c_double), ("lz", ctypes.c_double),
        ("y_stretch", ctypes.c_int), ("stretch_b", ctypes.c_double),
        ("bc_y", ctypes.c_int),
        ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("visc", ctypes.c_int),
        ("mu_ref", ctypes.c_double), ("T_ref", ctypes.c_double), ("visc_exp", ctypes.c_double),
        ("T_wall", ctypes.c_double), ("force_x", ctypes.c_double),
        ("recon", ctypes.c_int), ("flux", ctypes.c_int),
        ("tau_num_C", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("prec", ctypes.c_int),
        ("rho_ref", ctypes.c_double), ("p_ref", ctypes.c_double),
        ("force_mode", ctypes.c_int), ("mass_flux", ctypes.c_double),
        ("recon_vars", ctypes.c_int),
    ]


class HgksDiag(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("dt", ctypes.c_double),
        ("mass", ctypes.c_double), ("mom", ctypes.c_double * 3), ("energy", ctypes.c_double),
        ("Ek", ctypes.c_double), ("rho_min", ctypes.c_double), ("p_min", ctypes.c_double),
        ("step", ctypes.c_longlong), ("force_x", ctypes.c_double),
    ]


class HgksTurbulence(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "t", "Ek", "K", "zeta", "eps1", "eps2", "eps3", "rho_mean", "rho_rms", "u_rms", "Su", "Fu",
        "eps_s", "eps_d", "p_theta", "theta_rms", "omega_rms")] + [
        ("du2", ctypes.c_double * 3), ("du3", ctypes.c_double * 3), ("du4", ctypes.c_double * 3),
        ("eps_zeta", ctypes.c_double)]


class HgksHistoryRec(ctypes.Structure):
    _fields_ = [("s", HgksTurbulence), ("step", ctypes.c_longlong), ("eps_Ek", ctypes.c_double),
                ("eps_num", ctypes.c_double)]


class HgksChannel(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "t", "tau_w", "tau_w_lower", "tau_w_upper", "rho_w", "mu_w", "u_tau", "Re_tau",
        "U_b", "U_c", "rho_b", "Re_b", "Re_c", "C_f")]


_lock = threading.Lock()
_lib = None


class HgksError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load libhgks.so (built by paper_2005_08736_gb300.build); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library {p} is missing; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(p)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        pd = ctypes.POINTER(ctypes.c_double)
        pcfg = ctypes.POINTER(HgksConfig)
        L.hgks_default_config.argtypes = [pcfg, i]
        L.hgks_create.argtypes = [pcfg, vp, ctypes.POINTER(vp)]
        L.hgks_destroy.argtypes = [vp]
        L.hgks_init_state.argtypes = [vp, vp, i]
        L.hgks_init_conservative.argtypes = [vp, vp, i]
        L.hgks_get_state.argtypes = [vp, vp, i]
        L.hgks_step.argtypes = [vp, i, d, i, pd]
        L.hgks_diagnostics.argtypes = [vp, ctypes.POINTER(HgksDiag)]
        L.hgks_turbulence_stats.argtypes = [vp, ctypes.POINTER(HgksTurbulence)]
        L.hgks_profile_step.argtypes = [vp, d, pd, i]
        L.hgks_adjoint_step.argtypes = [vp, d, vp, vp]
        pi_ = ctypes.POINTER(ctypes.c_int)
        L.hgks_autotune.argtypes = [vp, pi_, pi_, pd]
        L.hgks_set_sweep_shape.argtypes = [vp, i, i]
        L.hgks_ensemble_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
        L.hgks_ensemble_step.argtypes = [vp, i, d, i]
        L.hgks_ensemble_destroy.argtypes = [vp]
        L.hgks_ensemble_set_batched.argtypes = [vp, i]
        L.hgks_ensemble_last_error.argtypes = [vp]
        L.hgks_ensemble_last_error.restype = ctypes.c_char_p
        L.hgks_step_noalloc.argtypes = [pcfg, vp, i, d, vp]
        L.hgks_measure_fp_peaks.argtypes = [vp, pd]
        L.hgks_channel_stats.argtypes = [vp, pd, ctypes.POINTER(HgksChannel)]
        L.hgks_set_time.argtypes = [vp, d, ctypes.c_longlong]
        L.hgks_count_flops.argtypes = [pcfg, i, pd]
        L.hgks_channel_compose.argtypes = [pcfg, pd, pd, ctypes.POINTER(HgksChannel)]
        L.hgks_cell_widths.argtypes = [pcfg, i, pd]
        L.hgks_kinetic_energy.argtypes = [vp, vp, vp, pd]
        L.hgks_history_start.argtypes = [vp, i, i]
        L.hgks_history_stop.argtypes = [vp]
        L.hgks_history_read.argtypes = [vp, ctypes.POINTER(HgksHistoryRec), i, ctypes.POINTER(i)]
        L.hgks_last_error.argtypes = [vp]
        L.hgks_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("hgks_last_error", "hgks_ensemble_last_error"):
                getattr(L, name).restype = i
        _lib = L
        return L


def check(status: int, ctx=None) -> None:
    if status != HGKS_OK:
        msg = load().hgks_last_error(ctx)
        raise HgksError(status, msg.decode() if msg else "")
