"""Python API over the C ABI: a GPU HGKS simulation on one device.

PyTorch provides the device memory for field transfers and the CUDA stream
the library runs on; every step of the scheme runs in the library's CUDA
kernels.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, fields

import numpy as np
import torch

from . import _lib

RECON = {"linear": 0, "weno-js": 1, "weno-z": 2}
FLUX = {"smooth": 0, "full": 1}
PREC = {"fp64": 0, "fp32": 1}


@dataclass
class Config:
    """Problem statement (mirrors hgks_config of include/hgks.h)."""
    nx: int
    ny: int
    nz: int
    x0: float = 0.0
    lx: float = 2 * math.pi
    y0: float = 0.0
    ly: float = 2 * math.pi
    z0: float = 0.0
    lz: float = 2 * math.pi
    y_stretch: int = 0
    stretch_b: float = 2.0
    bc_y: int = 0
    gamma: float = 1.4
    prandtl: float = 0.72
    visc: int = 0
    mu_ref: float = 1.0 / 1600.0
    T_ref: float = 1.0
    visc_exp: float = 0.76
    T_wall: float = 1.0
    force_x: float = 0.0
    recon: int = 0
    flux: int = 0
    tau_num_C: float = 0.0
    cfl: float = 0.5
    prec: int = 1
    rho_ref: float = 1.0
    p_ref: float = 100.0 / 1.4
    force_mode: int = 0       # 0 constant force_x; 1 constant mass flux (Sec. 3.3)
    mass_flux: float = 0.0    # force_mode 1: target volume average of rho U
    recon_vars: int = 0       # 1: WENO in characteristic variables (Sec. 2.1, Remark 1)

    def c_struct(self) -> _lib.HgksConfig:
        return _lib.HgksConfig(**{f.name: getattr(self, f.name) for f in fields(self)})

    @property
    def shape(self):
        return (5, self.nz, self.ny, self.nx)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def taylor_green_config(n: int, prec: str = "fp32", recon: str = "linear", flux: str = "smooth",
                        **kw) -> Config:
    """Taylor-Green vortex of Sec. 3.1: Ma 0.1, Re 1600 (mu = 1/1600), gamma 1.4."""
    c = Config(n, n, n, prec=PREC[prec], recon=RECON[recon], flux=FLUX[flux],
               tau_num_C=1.0 if flux == "full" else 0.0)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def isotropic_config(n: int, prec: str = "fp32", mach_t: float = 0.5, k0: float = 8.0,
                     recon: str = "weno-z", flux: str = "full", **kw) -> Config:
    """Decaying isotropic turbulence of Sec. 3.4 on [0, 2 pi]^3: Re_lambda 72,
    mu = mu0 (T/T0)^0.76, Pr 0.7, gamma 1.4, WENO-Z with the full flux and the
    numerical collision time; the initial constants (mu0, T0 = p0) from the
    spectrum E(k) = A0 k^4 exp(-2 k^2/k0^2) and Ma_t.  Start it with
    inputs.isotropic(n, seed, k0=k0, mach_t=mach_t)."""
    from . import inputs
    ic = inputs.isotropic_constants(k0=k0, mach_t=mach_t)
    c = Config(n, n, n, prec=PREC[prec], recon=RECON[recon], flux=FLUX[flux],
               tau_num_C=1.0 if flux == "full" else 0.0, prandtl=0.7, visc=1, mu_ref=ic["mu0"],
               T_ref=ic["T0"], visc_exp=0.76, p_ref=ic["p0"], rho_ref=1.0)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def channel_config(nx: int = 128, ny: int = 128, nz: int = 96, prec: str = "fp32", **kw) -> Config:
    """Turbulent channel of Sec. 3.3 at Re_tau 180: box 2 pi x 2 x pi, tanh
    stretching in y (b = 2), isothermal no-slip walls at y = -1, 1 with
    T_wall = c0^2/gamma (c0 = 10, bulk Ma 0.1), mu = 0.0541/180, constant
    streamwise force f_x = 2.93e-3, linear weights with the smooth flux.
    Start it with inputs.channel(nx, ny, nz, seed)."""
    c = Config(nx, ny, nz, lx=2 * math.pi, ly=2.0, y0=-1.0, lz=math.pi, y_stretch=1, stretch_b=2.0,
               bc_y=1, T_wall=100 / 1.4, mu_ref=0.0541 / 180, force_x=2.93e-3, prec=PREC[prec],
               recon=0, flux=0, prandtl=0.72)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


class Simulation:
    """One HGKS context on the current CUDA device."""

    def __init__(self, cfg: Config, stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.cfg = cfg
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._c = cfg.c_struct()
        h = ctypes.c_void_p()
        _lib.check(self.lib.hgks_create(ctypes.byref(self._c), ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hgks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, status):
        _lib.check(status, self.h)

    def _fp64_arg(self, a):
        """(pointer, is_host, keep-alive) for an FP64 [5][nz][ny][nx] array."""
        if isinstance(a, torch.Tensor):
            assert a.dtype == torch.float64 and tuple(a.shape) == self.cfg.shape
            a = a.contiguous()
            if a.is_cuda:
                # Order the caller's producer stream before the library's stream.
                self.stream.wait_stream(torch.cuda.current_stream(a.device))
                return ctypes.c_void_p(a.data_ptr()), 0, a
            return ctypes.c_void_p(a.data_ptr()), 1, a
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        assert arr.shape == self.cfg.shape
        return ctypes.c_void_p(arr.ctypes.data), 1, arr

    def init_primitive(self, prim) -> None:
        p, host, keep = self._fp64_arg(prim)
        self._call(self.lib.hgks_init_state(self.h, p, host))
        if not host:
            keep.record_stream(self.stream)

    def init_conservative(self, cons) -> None:
        p, host, keep = self._fp64_arg(cons)
        self._call(self.lib.hgks_init_conservative(self.h, p, host))
        if not host:
            keep.record_stream(self.stream)

    def step(self, nsteps: int = 1, dt: float = 0.0, sync: bool = True) -> float | None:
        t = ctypes.c_double(0.0)
        self._call(self.lib.hgks_step(self.h, int(nsteps), float(dt), int(sync), ctypes.byref(t)))
        return t.value if sync else None

    def state(self, device: bool = False, out=None):
        """Conservative state, FP64 [5][nz][ny][nx] (numpy, or a CUDA tensor).
        `out`: a host (e.g. pinned) FP64 CPU tensor of that shape to fill
        instead (returned)."""
        if out is not None:
            assert (isinstance(out, torch.Tensor) and not out.is_cuda and out.dtype == torch.float64
                    and tuple(out.shape) == self.cfg.shape and out.is_contiguous())
            self._call(self.lib.hgks_get_state(self.h, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        if device:
            out = torch.empty(self.cfg.shape, dtype=torch.float64, device=self.device)
            self._call(self.lib.hgks_get_state(self.h, ctypes.c_void_p(out.data_ptr()), 0))
            out.record_stream(self.stream)
            torch.cuda.current_stream(self.device).wait_stream(self.stream)
            return out
        out = np.empty(self.cfg.shape)
        self._call(self.lib.hgks_get_state(self.h, ctypes.c_void_p(out.ctypes.data), 1))
        return out

    def save_checkpoint(self, path: str) -> None:
        """Write the state (FP64 conservative), the time and the step counter
        to an .npz file."""
        d = self.diagnostics()
        np.savez(path, state=self.state(), t=d["t"], step=d["step"],
                 shape=np.array(self.cfg.shape))

    def load_checkpoint(self, path: str) -> None:
        """Resume from save_checkpoint's file (same grid): the state, the
        time and the step counter.  In FP32 the accumulation's compensation
        restarts at zero."""
        ck = np.load(path)
        if tuple(ck["shape"]) != tuple(self.cfg.shape):
            raise ValueError(f"checkpoint grid {tuple(ck['shape'])} != {self.cfg.shape}")
        self.init_conservative(ck["state"])
        self._call(self.lib.hgks_set_time(self.h, float(ck["t"]), int(ck["step"])))

    def adjoint_step(self, dt: float, adj_in: torch.Tensor, adj_out: torch.Tensor) -> None:
        """adj_out = (dQ^{n+1}/dQ^n)^T adj_in at the current state Q^n (device FP64 tensors)."""
        for t in (adj_in, adj_out):
            assert t.is_cuda and t.dtype == torch.float64 and tuple(t.shape) == self.cfg.shape
            assert t.is_contiguous()
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._call(self.lib.hgks_adjoint_step(self.h, float(dt), ctypes.c_void_p(adj_in.data_ptr()),
                                              ctypes.c_void_p(adj_out.data_ptr())))
        adj_in.record_stream(self.stream)
        adj_out.record_stream(self.stream)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def autotune(self, cache: str | None = None) -> dict:
        """Pick the sweep's launch shape for this configuration (tile variant and
        face layers per CTA) by timing the candidates on the current state; with
        `cache` (a JSON file) a known configuration reuses its stored choice."""
        import json
        import os
        key = json.dumps({f.name: getattr(self.cfg, f.name) for f in fields(self.cfg)},
                         sort_keys=True)
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
        if key in table:
            v, c = table[key]["variant"], table[key]["chunk"]
            self._call(self.lib.hgks_set_sweep_shape(self.h, int(v), int(c)))
            return dict(table[key], cached=True)
        v, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._call(self.lib.hgks_autotune(self.h, ctypes.byref(v), ctypes.byref(c), ctypes.byref(ms)))
        rec = {"variant": v.value, "chunk": c.value, "sweep_ms": ms.value}
        if cache:
            table[key] = rec
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1)
            os.replace(tmp, cache)
        return dict(rec, cached=False)

    def profile_step(self, dt: float = 0.0) -> dict:
        """Advance one step with CUDA events per kernel class; device ms per class."""
        ms = (ctypes.c_double * len(_lib.KERNEL_CLASSES))()
        self._call(self.lib.hgks_profile_step(self.h, float(dt), ms, len(ms)))
        return dict(zip(_lib.KERNEL_CLASSES, list(ms)))

    def diagnostics(self) -> dict:
        d = _lib.HgksDiag()
        self._call(self.lib.hgks_diagnostics(self.h, ctypes.byref(d)))
        return dict(t=d.t, dt=d.dt, mass=d.mass, mom=tuple(d.mom), energy=d.energy, Ek=d.Ek,
                    rho_min=d.rho_min, p_min=d.p_min, step=d.step, force_x=d.force_x)

    def turbulence(self) -> dict:
        """Turbulence statistics of the current state (Sec. 3.1, Sec. 3.4):
        E_k, K, enstrophy zeta, eps1..eps3, rho_rms, u_rms, S_u, F_u, eps_s,
        eps_d, <p theta> and the per-axis moments du{2,3,4}_{x,y,z}."""
        d = _lib.HgksTurbulence()
        self._call(self.lib.hgks_turbulence_stats(self.h, ctypes.byref(d)))
        return _turb_dict(d)

    def history_start(self, every: int, capacity: int = 4096) -> None:
        """Record the statistics of the current state and, every `every`
        steps, of the stepped state (on the device, inside the step)."""
        self._call(self.lib.hgks_history_start(self.h, int(every), int(capacity)))

    def history_stop(self) -> None:
        self._call(self.lib.hgks_history_stop(self.h))

    def history(self) -> list:
        """The recorded statistics, oldest first: each a dict of the
        turbulence statistics with step, eps_Ek = -dE_k/dt and
        eps_num = eps_Ek - (eps1 + eps2 + eps3) (Sec. 3.1)."""
        n = ctypes.c_int()
        self._call(self.lib.hgks_history_read(self.h, None, 0, ctypes.byref(n)))
        recs = (_lib.HgksHistoryRec * max(n.value, 1))()
        self._call(self.lib.hgks_history_read(self.h, recs, n.value, ctypes.byref(n)))
        return [dict(_turb_dict(r.s), step=r.step, eps_Ek=r.eps_Ek, eps_num=r.eps_num)
                for r in recs[:n.value]]

    def channel_stats(self) -> dict:
        """Mean-flow statistics of the wall-bounded channel (Sec. 3.3,
        hgks_channel_stats): tau_w, u_tau, Re_tau, U_b, U_c, Re_b, Re_c, C_f,
        the plane-mean profiles per y row ("profiles"), and the library's
        wall-unit profiles y, y_plus, U_plus, uv_plus, dUp_dYp and the
        total-stress residual."""
        out = _lib.HgksChannel()
        ny = self.cfg.ny
        prof = np.empty((len(_lib.CHANNEL_PROFILES), ny))
        self._call(self.lib.hgks_channel_stats(
            self.h, prof.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(out)))
        res = {k: getattr(out, k) for k, _ in _lib.HgksChannel._fields_}
        res["profiles"] = dict(zip(_lib.CHANNEL_PROFILES[:8], prof[:8]))
        for name, row in zip(_lib.CHANNEL_PROFILES[8:], prof[8:]):
            res[name] = row
        return res

    def kinetic_energy(self, q: torch.Tensor, grad: torch.Tensor | None = None) -> float:
        """E_k of Sec. 3.1 of an FP64 conservative device tensor
        [5][nz][ny][nx] (hgks_kinetic_energy); with `grad` (same shape) also
        dE_k/dQ."""
        for t in (q,) if grad is None else (q, grad):
            assert t.is_cuda and t.dtype == torch.float64 and tuple(t.shape) == self.cfg.shape
            assert t.is_contiguous()
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        ek = ctypes.c_double()
        self._call(self.lib.hgks_kinetic_energy(
            self.h, ctypes.c_void_p(q.data_ptr()),
            ctypes.c_void_p(grad.data_ptr() if grad is not None else None), ctypes.byref(ek)))
        q.record_stream(self.stream)
        if grad is not None:
            grad.record_stream(self.stream)
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return ek.value


def _turb_dict(d) -> dict:
    out = {k: getattr(d, k) for k, _ in d._fields_ if not k.startswith("du")}
    for k in ("du2", "du3", "du4"):
        for i, a in enumerate("xyz"):
            out[f"{k}_{a}"] = getattr(d, k)[i]
    return out


def cell_widths(cfg: Config, axis: int) -> np.ndarray:
    """Cell widths along axis 0, 1, 2 of the grid cfg describes
    (hgks_cell_widths: uniform, or the tanh mapping of Sec. 3.3 in y)."""
    lib = _lib.load()
    n = (cfg.nx, cfg.ny, cfg.nz)[axis]
    out = np.empty(n)
    c = cfg.c_struct()
    _lib.check(lib.hgks_cell_widths(ctypes.byref(c), int(axis),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


class Ensemble:
    """Independent simulations advanced by one CUDA graph launch per step:
    one batched kernel launch per phase for all members when they share a
    scheme (the default then), else every member's launches as parallel graph
    branches.  batched=False forces the branches; batched=True requires the
    batched form."""

    def __init__(self, sims: list, batched: bool | None = None):
        self.lib = _lib.load()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(sims))(*[s.h.value for s in sims])
        h = ctypes.c_void_p()
        _lib.check(self.lib.hgks_ensemble_create(arr, len(sims), ctypes.byref(h)))
        self.h = h
        if batched is not None:
            status = self.lib.hgks_ensemble_set_batched(self.h, int(bool(batched)))
            if status != _lib.HGKS_OK:
                msg = self.lib.hgks_ensemble_last_error(self.h)
                raise _lib.HgksError(status, msg.decode() if msg else "")

    def step(self, nsteps: int = 1, dt: float = 0.0, sync: bool = True) -> None:
        status = self.lib.hgks_ensemble_step(self.h, int(nsteps), float(dt), int(sync))
        if status != _lib.HGKS_OK:
            msg = self.lib.hgks_ensemble_last_error(self.h)
            raise _lib.HgksError(status, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.hgks_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StepWindow(torch.autograd.Function):
    """Q^0 -> Q^K by K steps of fixed dt, differentiable through the library's
    adjoint step.  The forward keeps a checkpoint every `every` steps; the
    backward recomputes each window from its checkpoint and applies the
    adjoint steps in reverse.  Tensors are device FP64 conservative states
    [5][nz][ny][nx]."""

    @staticmethod
    def forward(ctx, q0, sim: "Simulation", nsteps: int, dt: float, every: int):
        sim.init_conservative(q0.detach())
        ckpts = {}
        for n in range(nsteps):
            if n % every == 0:
                ckpts[n] = sim.state(device=True).clone()
            sim.step(1, dt)
        ctx.sim, ctx.nsteps, ctx.dt, ctx.every, ctx.ckpts = sim, nsteps, dt, every, ckpts
        return sim.state(device=True)

    @staticmethod
    def backward(ctx, grad):
        sim, dt = ctx.sim, ctx.dt
        lam = grad.detach().contiguous().to(torch.float64)
        for start in sorted(ctx.ckpts, reverse=True):
            end = min(start + ctx.every, ctx.nsteps)
            states = []
            sim.init_conservative(ctx.ckpts[start])
            for n in range(start, end):
                states.append(sim.state(device=True).clone())
                if n < end - 1:
                    sim.step(1, dt)
            for n in range(end - 1, start - 1, -1):
                sim.init_conservative(states[n - start])
                out = torch.empty_like(lam)
                sim.adjoint_step(dt, lam, out)
                lam = out
        return lam, None, None, None, None


def run_window(q0: torch.Tensor, sim: Simulation, nsteps: int, dt: float, every: int = 10):
    """Differentiable K-step map (see StepWindow)."""
    return StepWindow.apply(q0, sim, nsteps, dt, every)


class _KineticEnergy(torch.autograd.Function):
    """E_k of a device state through hgks_kinetic_energy; its gradient is the
    library's dE_k/dQ."""

    @staticmethod
    def forward(ctx, q, sim: "Simulation"):
        q = q.detach().contiguous()
        grad = torch.empty_like(q)
        ek = sim.kinetic_energy(q, grad)
        ctx.save_for_backward(grad)
        return torch.tensor(ek, dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None


def kinetic_energy(q: torch.Tensor, sim: "Simulation") -> torch.Tensor:
    """E_k = (1/(rho_ref |Omega|)) sum rho |U|^2 / 2 |Omega_c| (Sec. 3.1) of a
    device FP64 conservative state, differentiable (the library computes the
    value and dE_k/dQ on the device)."""
    return _KineticEnergy.apply(q, sim)


def total_stress_residual(stats: dict) -> tuple[np.ndarray, np.ndarray]:
    """The stationarity check of the channel (Sec. 3.3) on the lower half of
    the channel: (Y+, dU+/dY+ - <u'v'>+ - (1 - Y+/Re_tau)) from the profiles
    hgks_channel_stats computes (Simulation.channel_stats)."""
    y = stats["y"]
    lower = y < y[0] + 0.5 * (y[-1] - y[0]) + 1e-12
    return stats["y_plus"][lower], stats["total_stress_residual"][lower]


def measure_fp_peaks(stream: torch.cuda.Stream | None = None) -> dict:
    """Measured FMA throughput of the current GPU in TFLOP/s: FP32, packed
    FP32 pairs and FP64 (hgks_measure_fp_peaks)."""
    lib = _lib.load()
    out = (ctypes.c_double * 3)()
    s = stream if stream is not None else torch.cuda.current_stream()
    _lib.check(lib.hgks_measure_fp_peaks(ctypes.c_void_p(s.cuda_stream), out))
    return {"fp32": out[0], "fp32x2": out[1], "fp64": out[2]}
