"""Throughput of the HGKS S2O4 step on the GPU (Mcell-updates/s).

Workload: the Taylor-Green vortex of Cao, Pan & Xu (arXiv:2005.08736,
Sec. 3.1) on a 256^3 periodic grid -- Ma 0.1, Re 1600, gamma 1.4, Pr 0.72 --
with linear-weight WENO5 and the smooth BGK flux (the paper's setting for this
flow), CFL 0.5, FP32 arithmetic with deviation storage and FP64 reductions.
One "step" is one full S2O4 time step (CFL reduction, two stages of ghost
fill, reconstruction, Gauss-point flux and update).  The same step in FP64 is
timed beside it, with the FP32-vs-FP64 error after the timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (the
domain-decomposed multi-GPU path is not built); value = sum over ranks.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 256
PAPER_MCUPS_256 = 2.0 ** 24 / 9.09 / 1e6  # Sec. 3.2 table: 256^3, 64 cores, 9.09 s/step
METRIC = "Mcell-updates/s per S2O4 step"
# cfl, dt, 2 x (3 ghost fills + transposed copy + 3 sweeps + update), time
LAUNCHES_PER_STEP = 19
# Algorithmic work of the sweep kernel per face comes from hgks_count_flops:
# the kernel's closed forms run on the host with a counting number type, for
# one face point's face fields, one point's t1 pass and one face's t2 pass and
# flux -- i.e. without the tile's halo recomputation -- with common
# subexpressions counted once and dead results not counted (additions,
# multiplications and divisions; square roots, exponentials and error
# functions are listed beside it, not counted as flops).
# Algorithmic HBM bytes of one FP32 step per cell: stage 1 reads Q^n and
# writes Q* and the increment, stage 2 reads Q* and the increment and writes
# Q^{n+1}: 6 x 5 x 4 B.
ALG_BYTES_PER_CELL_STEP = 120.0
# Per tile variant: EXECUTED FP32 flops per face (fadd + fmul + 2 ffma, mean
# of the three directions, ncu at 128^3, halo recomputation and the
# polynomial evaluation of erf/exp included; the packed variant performs the
# operations of variant 1) and DRAM bytes (read + write) per face of the
# stage-1 sweep from a one-pass ncu capture at 256^3 (None where not captured
# for the current kernel; at 128^3 the L2 holds part of the writes, so
# smaller grids undercount).  Reported beside the algorithmic count.
SWEEP_COUNTS = {0: {"tile": "16x8, 4 layers", "flops": 2391.8, "dram": None},
                1: {"tile": "32x8, 2 layers", "flops": 2313.7, "dram": None},
                2: {"tile": "16x16, 2 layers", "flops": 2247.7, "dram": None},
                3: {"tile": "32x8, 2 layers, packed FP32 pairs", "flops": 2313.7, "dram": 58.3}}


def alg_flops_per_face(cfg, stage: int = 1) -> dict:
    """Algorithmic operations of one face of the sweep kernel for `cfg`
    (hgks_count_flops): flops = additions + multiplications + divisions of the
    face fields (one point), the t1 pass (one point) and the t2 pass and flux
    (one face); the transcendental calls listed beside them."""
    import ctypes
    from paper_2005_08736_gb300 import _lib
    lib = _lib.load()
    out = (ctypes.c_double * 21)()
    c = cfg.c_struct()
    _lib.check(lib.hgks_count_flops(ctypes.byref(c), int(stage), out))
    names = ("add", "mul", "div", "sqrt", "exp", "erf", "pow")
    parts = [dict(zip(names, out[7 * k:7 * k + 7])) for k in range(3)]
    fl = [p["add"] + p["mul"] + p["div"] for p in parts]
    return {"flops": sum(fl), "face_fields": fl[0], "t1_pass": fl[1], "t2_flux": fl[2],
            "transcendentals": {k: sum(p[k] for p in parts) for k in ("sqrt", "exp", "erf", "pow")}}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi SM clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_sample(steps: int = 1, n: int = 32, seconds: float = 0.0):
    """The FP64 oracle on a bounded sample of the workload: Taylor-Green n^3
    from its initial state, `steps` steps, or whole steps until `seconds` have
    elapsed (at least one); (Mcell-upd/s, seconds, steps)."""
    import oracle
    from paper_2005_08736_gb300 import inputs
    s = oracle.Solver(oracle.Config(n, n, n, recon=0, flux=0, prandtl=0.72, mu_ref=1 / 1600,
                                    cfl=0.5))
    s.set_state(oracle.conservative(inputs.taylor_green(n), 1.4))
    done, el = 0, 0.0
    t0 = time.perf_counter()
    while done < steps or el < seconds:
        s.step(1)
        done += 1
        el = time.perf_counter() - t0
    return n ** 3 * done / el / 1e6, el, done


def oracle_threads() -> int:
    import oracle
    return oracle.threads()


def oracle_sample_one_core(n: int = 32):
    """oracle_sample(1, n) in a child process restricted to one OpenMP thread;
    (Mcell-upd/s, seconds)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = f"import bench, json; print(json.dumps(bench.oracle_sample(1, {n})))"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600, check=True)
    rate, secs, _ = json.loads(out.stdout.strip().splitlines()[-1])
    return rate, secs


# The reference arm's whole run (warm-up and timed steps) is held to about
# this many seconds by shrinking each step's sample grid.
REFERENCE_RUN_SECONDS = 150.0


def run_reference(args, rank: int):
    if rank != 0:
        return
    import oracle
    oracle.build()
    # One step of the 32^3 sample loads the library and gives the time per
    # step; a smaller grid is taken if K + W such steps would exceed the bound.
    n = 32
    _, t_step, _ = oracle_sample(1, n)
    while n > 16 and (args.steps + args.warmup) * t_step > REFERENCE_RUN_SECONDS:
        t_step *= ((n - 8) / n) ** 3
        n -= 8
    for _ in range(args.warmup):
        oracle_sample(1, n)
    rates, times = [], []
    for _ in range(args.steps):
        r, el, _ = oracle_sample(1, n)
        rates.append(r)
        times.append(el)
    value = n ** 3 * args.steps / sum(times) / 1e6
    cores = oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mcell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config_dict(), sample_grid=[n] * 3, sample_precision="fp64",
                       sample_note=f"each timed step is one FP64 oracle step of the same "
                                   f"Taylor-Green workload on a {n}^3 grid"),
        "cpu_baseline": {"value": value, "unit": "Mcell-updates/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"FP64 CPU oracle, one step of Taylor-Green {n}^3 per timed step "
                                   f"(same physics and scheme as the {N_GRID}^3 workload)"},
        "e2e": {"value": value, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def adjoint_ratio(prec: int, flux: int, reps: int = 5) -> dict:
    """Adjoint step / forward step at 64^3 (isotropic, kappa0 = 4, Ma_t 0.5,
    WENO-Z, power-law viscosity, numerical collision time), dt fixed."""
    import torch
    from paper_2005_08736_gb300 import inputs
    from paper_2005_08736_gb300.solver import Config, Simulation

    c = inputs.isotropic_constants(k0=4.0, mach_t=0.5)
    cfg = Config(64, 64, 64, prec=prec, recon=2, flux=flux, tau_num_C=1.0, prandtl=0.7, visc=1,
                 mu_ref=c["mu0"], T_ref=c["T0"], visc_exp=0.76, p_ref=c["p0"], rho_ref=1.0)
    sim = Simulation(cfg)
    sim.init_primitive(inputs.isotropic(64, 0, k0=4.0))
    dt = 2e-3  # a fixed step (the timing does not depend on its size)

    def timed(fn, n):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / n

    sim.step(2, dt)
    fwd = timed(lambda: sim.step(1, dt, sync=False), 2 * reps)
    lam = torch.randn(cfg.shape, dtype=torch.float64, device="cuda")
    o = torch.empty_like(lam)
    sim.adjoint_step(dt, lam, o)
    adj = timed(lambda: sim.adjoint_step(dt, lam, o), reps)
    sim.close()
    return {"forward_ms": 1e3 * fwd, "adjoint_ms": 1e3 * adj, "adjoint_over_forward": adj / fwd}


def run_adjoint(args):
    """--adjoint: the 64^3 adjoint / forward ratios (full and smooth flux, FP32
    and FP64); with --quick only --precision and --flux, one adjoint step
    after one warm-up (for profiling)."""
    from paper_2005_08736_gb300 import build
    build.build()
    if args.quick:
        prec = 1 if args.precision == "fp32" else 0
        flux = 1 if args.flux == "full" else 0
        print(json.dumps({f"adjoint_64_wenoz_{args.flux}_{args.precision}": adjoint_ratio(prec, flux, 1)}))
        return
    out = {}
    for flux, fname in ((1, "full"), (0, "smooth")):
        for prec, pname in ((1, "fp32"), (0, "fp64")):
            out[f"adjoint_64_wenoz_{fname}_{pname}"] = adjoint_ratio(prec, flux)
    print(json.dumps(out, indent=1))


def extra_workloads(steps: int, peak_tflops: float | None = None):
    """The other measured configurations: isotropic turbulence 256^3 (WENO-Z +
    full flux, FP32), the stretched wall-bounded channel 128 x 128 x 96 (FP32),
    the adjoint / forward time ratio at 64^3 (isotropic, kappa0 = 4, WENO-Z +
    full flux, FP64 and FP32), and an ensemble of 24 isotropic instances of
    mixed sizes in one graph launch per step against sequential runs."""
    import torch
    from paper_2005_08736_gb300 import inputs
    from paper_2005_08736_gb300.solver import Config, Ensemble, Simulation

    def timed(fn, reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    out = {}
    # Isotropic turbulence (Sec. 3.4): Ma_t 0.5, Re_lambda 72, mu ~ T^0.76, Pr 0.7.
    def iso_cfg(n, prec, k0=8.0):
        c = inputs.isotropic_constants(k0=k0, mach_t=0.5)
        return Config(n, n, n, prec=prec, recon=2, flux=1, tau_num_C=1.0, prandtl=0.7, visc=1,
                      mu_ref=c["mu0"], T_ref=c["T0"], visc_exp=0.76, p_ref=c["p0"], rho_ref=1.0)
    cfg = iso_cfg(256, 1)
    sim = Simulation(cfg)
    sim.init_primitive(inputs.isotropic(256, 0))
    iso_tune = sim.autotune()
    sim.step(3)
    s_per = timed(lambda: sim.step(steps, sync=False), 1) / steps
    prof = sim.profile_step()
    # ALU roofline of its stage-1 sweep: algorithmic flops per face (the
    # kernel's formulas, hgks_count_flops) x faces per launch / launch time.
    alg = alg_flops_per_face(cfg, 1)
    faces = (cfg.nx + 1) * cfg.ny * cfg.nz
    launch_ms = prof["flux_stage1"] / 3.0
    achieved = alg["flops"] * faces / (launch_ms * 1e-3) / 1e12
    out["isotropic_256_wenoz_full_fp32"] = {
        "ms_per_step": 1e3 * s_per, "mcups": cfg.cells / s_per / 1e6,
        "kernel_ms_per_step": prof, "autotune": iso_tune,
        "roofline": {"bound": "alu", "kernel": "k_sweep stage 1 (FP32, WENO-Z, full flux)",
                     "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops if peak_tflops else None,
                     "alg_flops_per_face": alg, "launch_ms": launch_ms,
                     "peak_source": "measured FP32 FMA throughput of this GPU"}}
    sim.close()
    # Channel (Sec. 3.3): 128 x 128 x 96, tanh b = 2, walls, f_x = 2.93e-3, Ma 0.1.
    ccfg = Config(128, 128, 96, lx=2 * 3.141592653589793, ly=2.0, y0=-1.0, lz=3.141592653589793,
                  y_stretch=1, stretch_b=2.0, bc_y=1, T_wall=100 / 1.4, mu_ref=0.0541 / 180,
                  force_x=2.93e-3, prec=1, recon=0, flux=0, prandtl=0.72)
    sim = Simulation(ccfg)
    sim.init_primitive(inputs.channel(128, 128, 96, 0))
    ch_tune = sim.autotune()
    sim.step(3)
    s_per = timed(lambda: sim.step(steps, sync=False), 1) / steps
    out["channel_128x128x96_fp32"] = {"ms_per_step": 1e3 * s_per,
                                      "mcups": ccfg.cells / s_per / 1e6, "autotune": ch_tune}
    sim.close()
    # Adjoint / forward time ratio at 64^3.
    for prec, name in ((0, "fp64"), (1, "fp32")):
        out[f"adjoint_64_wenoz_full_{name}"] = adjoint_ratio(prec, 1)
    # Ensemble of 24 isotropic instances, grids {32, 48, 64, 96}^3 by seed, FP32.
    sims, cells = [], 0
    for seed in range(24):
        n = (32, 48, 64, 96)[seed % 4]
        sim = Simulation(iso_cfg(n, 1))
        sim.init_primitive(inputs.isotropic(n, seed))
        sims.append(sim)
        cells += n ** 3
    ens = Ensemble(sims)  # batched: one launch per phase for all 24 members
    ens.step(2)
    t_ens = timed(lambda: ens.step(steps, sync=False), 1) / steps
    # The same batch as graph branches (each member's own launches).
    ensb = Ensemble(sims, batched=False)
    ensb.step(2)
    t_br = timed(lambda: ensb.step(steps, sync=False), 1) / steps
    ensb.close()
    # Sequential runs: each member advanced alone, one after another.
    t_seq = timed(lambda: [s.step(steps, sync=True) for s in sims], 1) / steps
    # Each member's own graph launched on its own stream without waiting (the
    # streams may overlap on the device).
    t_str = timed(lambda: [s.step(steps, sync=False) for s in sims], 1) / steps
    out["ensemble_24_isotropic_mixed"] = {
        "instances": 24, "cells": cells, "ensemble_ms_per_step": 1e3 * t_ens,
        "sequential_ms_per_step": 1e3 * t_seq, "speedup": t_seq / t_ens,
        "member_streams_ms_per_step": 1e3 * t_str, "speedup_vs_member_streams": t_str / t_ens,
        "graph_branches_ms_per_step": 1e3 * t_br, "speedup_vs_graph_branches": t_br / t_ens,
        "launches_per_step": {"batched": LAUNCHES_PER_STEP, "branches": LAUNCHES_PER_STEP * 24},
        "ensemble_mcups": cells / t_ens / 1e6}
    ens.close()
    for s in sims:
        s.close()
    return out


def run_history(args):
    """Taylor-Green to t = 10 (Sec. 3.1) in FP32 and FP64 with the same fixed
    dt: the library's statistics history (recorded on the device every 10
    steps) -- E_k, eps(E_k) = -dE_k/dt by second-order differences, eps(zeta),
    eps1..eps3 and the numerical dissipation eps_num -- and the FP32 errors
    against the FP64 path (itself checked against the oracle).  --grid 128 by
    default; --t-end-fp64 stops the FP64 run earlier (the FP32 errors are then
    taken over the common interval, the density error at its end)."""
    import numpy as np
    from paper_2005_08736_gb300 import inputs
    from paper_2005_08736_gb300.solver import Simulation, taylor_green_config
    n, t_end, every = args.grid if args.grid_given else 128, args.t_end, 10
    prim = inputs.taylor_green(n)
    dt = 0.5 * (2 * np.pi / n) / 11.0  # CFL 0.5 with max(|u| + c) = 11 (Sec. 3.2 table)
    nsteps = int(round(t_end / dt))
    t64 = min(t_end, args.t_end_fp64) if args.t_end_fp64 else t_end
    nsteps64 = min(int(round(t64 / dt / every)) * every, nsteps // every * every)
    keys = ("t", "Ek", "zeta", "eps1", "eps2", "eps3", "eps_zeta", "eps_Ek", "eps_num")
    hist, finals, times = {}, {}, {}
    for prec in ("fp64", "fp32"):
        sim = Simulation(taylor_green_config(n, prec))
        sim.init_primitive(prim)
        total = nsteps64 if prec == "fp64" else nsteps
        sim.history_start(every, capacity=total // every + 2)
        t0 = time.perf_counter()
        done = 0
        while done < total:
            k = min(500, total - done)
            if done < nsteps64 <= done + k:
                k = nsteps64 - done
            sim.step(k, dt, sync=False)
            done += k
            if done == nsteps64:
                finals[prec] = sim.state()
        sim.step(0, dt)  # synchronise and check
        times[prec] = time.perf_counter() - t0
        recs = sim.history()
        hist[prec] = {key: np.array([r[key] for r in recs]) for key in keys}
        sim.close()
    h32, h64 = hist["fp32"], hist["fp64"]
    m = len(h64["t"])
    assert np.allclose(h32["t"][:m], h64["t"], rtol=1e-12, atol=0)

    def rel(key, scale_by_peak):
        a, b = h32[key][:m], h64[key]
        if not scale_by_peak:
            return float(np.max(np.abs(a - b) / np.abs(b)))
        # the differences of the FP32 E_k samples at the ends of a shortened
        # FP64 run are one-sided: compare the interior
        lo, hi = (1, m - 1) if m < len(h32["t"]) else (0, m)
        return float(np.max(np.abs(a[lo:hi] - b[lo:hi])) / np.max(np.abs(b)))
    a, b = finals["fp32"], finals["fp64"]
    rho_err = float(np.abs(a[0] - b[0]).max() / np.abs(b[0]).max())
    ipk = int(np.argmax(h32["eps_Ek"]))
    sub = slice(None, None, 10)
    out = {"workload": f"taylor-green-{n}^3 to t={t_end} (FP64 to t={nsteps64 * dt:.3f})",
           "steps": nsteps, "steps_fp64": nsteps64, "dt": dt, "samples_every_steps": every,
           "fp32_vs_fp64": {
               "Ek_rel_err_max": rel("Ek", False),
               "eps_Ek_err_max_of_peak": rel("eps_Ek", True),
               "eps_zeta_err_max_of_peak": rel("eps_zeta", True),
               "eps_num_err_max_of_peak_eps": float(
                   np.max(np.abs(h32["eps_num"][1:m - 1] - h64["eps_num"][1:m - 1])) / np.max(np.abs(h64["eps_Ek"]))),
               "rho_rel_linf_at_fp64_end": rho_err},
           "fp32": {"Ek_final": float(h32["Ek"][-1]), "eps_Ek_peak": float(h32["eps_Ek"][ipk]),
                    "t_eps_Ek_peak": float(h32["t"][ipk]), "eps_zeta_peak": float(h32["eps_zeta"].max()),
                    "eps_num_at_eps_peak": float(h32["eps_num"][ipk]),
                    "eps1_at_eps_peak": float(h32["eps1"][ipk])},
           "wall_s": times,
           "history_fp32_every_100_steps": {key: [float(x) for x in h32[key][sub]] for key in keys},
           "history_fp64_every_100_steps": {key: [float(x) for x in h64[key][sub]] for key in keys}}
    print(json.dumps(out), flush=True)


def run_errors(args):
    """FP32 against FP64 (same initial state, same fixed dt) for the isotropic
    (64^3, kappa0 = 4, Ma_t 0.5, WENO-Z + full flux) and channel (64x64x48,
    walls, stretched y, body force) workloads: relative L-inf per variable and
    the kinetic-energy error after `steps` steps."""
    import numpy as np
    from paper_2005_08736_gb300 import inputs
    from paper_2005_08736_gb300.solver import Config, Simulation
    out = {}
    c = inputs.isotropic_constants(k0=4.0, mach_t=0.5)
    cases = {
        "isotropic_64_wenoz_full": (
            lambda prec: Config(64, 64, 64, prec=prec, recon=2, flux=1, tau_num_C=1.0, prandtl=0.7,
                                visc=1, mu_ref=c["mu0"], T_ref=c["T0"], visc_exp=0.76,
                                p_ref=c["p0"]),
            inputs.isotropic(64, 0, k0=4.0), 0.5 * (2 * np.pi / 64) / (c["c0"] * 1.5)),
        "channel_64x64x48_linear_smooth": (
            lambda prec: Config(64, 64, 48, lx=2 * np.pi, ly=2.0, y0=-1.0, lz=np.pi, y_stretch=1,
                                stretch_b=2.0, bc_y=1, T_wall=100 / 1.4, mu_ref=0.0541 / 180,
                                force_x=2.93e-3, prec=prec, recon=0, flux=0),
            inputs.channel(64, 64, 48, 0), 2e-4),
    }
    for name, (mk, prim, dt) in cases.items():
        res = {}
        for prec in (0, 1):
            sim = Simulation(mk(prec))
            sim.init_primitive(prim)
            sim.step(args.steps, dt)
            res[prec] = (sim.state(), sim.diagnostics()["Ek"])
            sim.close()
        a, b = res[1][0], res[0][0]
        out[name] = {"steps": args.steps, "dt": dt,
                     "rel_linf": [float(np.abs(a[v] - b[v]).max() / np.abs(b[v]).max()) for v in range(5)],
                     "Ek_rel_err": abs(res[1][1] - res[0][1]) / res[0][1]}
    print(json.dumps(out), flush=True)


def run_gradcheck(args):
    """Gradient of the kinetic energy E_k after 50 steps with respect to the
    initial velocity of a 64^3 isotropic field (kappa0 = 4, Ma_t 0.5, seed 0,
    full flux, fixed dt; WENO-Z with the numerical collision time by default,
    --recon / --tau-num select others), in FP64 and FP32, through the autograd
    window with a checkpoint every 10 steps; checked against central
    differences of the FP64 forward step along 16 seeded unit directions
    (seeds 100-115), h = 1e-6 |u0| (and h / 10 along the first four, to show
    the convergence across the kinks of WENO-Z and |p_l - p_r|)."""
    import numpy as np
    import torch
    from paper_2005_08736_gb300 import inputs
    from paper_2005_08736_gb300.solver import Config, Simulation, kinetic_energy, run_window
    n, K, every, gamma = 64, 50, 10, 1.4
    c = inputs.isotropic_constants(k0=4.0, mach_t=0.5)
    prim = torch.from_numpy(inputs.isotropic(n, 0, k0=4.0)).cuda()
    dt = 0.5 * (2 * np.pi / n) / (c["c0"] * 1.5)

    recon = {"linear": 0, "weno-js": 1, "weno-z": 2}[args.recon if args.recon != "linear" else "weno-z"]
    C = 1.0 if args.tau_num is None else args.tau_num

    def cfg(prec):
        return Config(n, n, n, prec=prec, recon=recon, flux=1, tau_num_C=C, prandtl=0.7, visc=1,
                      mu_ref=c["mu0"], T_ref=c["T0"], visc_exp=0.76, p_ref=c["p0"], rho_ref=1.0)

    def cons(u):
        rho, p = prim[0], prim[4]
        return torch.stack([rho, rho * u[0], rho * u[1], rho * u[2],
                            p / (gamma - 1) + 0.5 * rho * (u * u).sum(0)])

    u0 = prim[1:4].clone()
    out = {"workload": f"isotropic-64^3 kappa0=4 Ma_t=0.5 recon={recon} full flux tau_num_C={C}, "
                       "E_k after 50 steps", "dt": dt, "checkpoint_every": every}
    grads = {}
    for prec, name in ((0, "fp64"), (1, "fp32")):
        sim = Simulation(cfg(prec))
        x = u0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = kinetic_energy(run_window(cons(x), sim, K, dt, every), sim)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        (g,) = torch.autograd.grad(J, x)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        grads[name] = g
        out[name] = {"J": J.item(), "forward_s": t1 - t0, "backward_s": t2 - t1,
                     "backward_over_forward": (t2 - t1) / (t1 - t0)}
        if prec == 0:
            fsim = sim
        else:
            sim.close()
    g64, g32 = grads["fp64"], grads["fp32"]
    out["fp32_grad_rel_linf_vs_fp64"] = ((g32 - g64).abs().max() / g64.abs().max()).item()

    def J_of(u):
        fsim.init_conservative(cons(u))
        fsim.step(K, dt)
        return kinetic_energy(fsim.state(device=True), fsim).item()

    unorm = u0.norm().item()
    h0 = 1e-6 * unorm
    # --fd-scales: the step sizes h / |u0| of the central differences along
    # every direction (default: 1e-6, and 1e-7 along the first four).
    scales = [float(x) for x in args.fd_scales.split(",")] if args.fd_scales else None
    rows = []
    for k, seed in enumerate(range(100, 116)):
        gen = torch.Generator(device="cuda").manual_seed(seed)
        v = torch.randn(u0.shape, dtype=torch.float64, device="cuda", generator=gen)
        v /= v.norm()
        ad64, ad32 = (g64 * v).sum().item(), (g32 * v).sum().item()
        row = {"seed": seed, "adjoint_fp64": ad64, "adjoint_fp32": ad32}
        hs = [sc * unorm for sc in scales] if scales else ((h0, h0 / 10) if k < 4 else (h0,))
        for h in hs:
            fd = (J_of(u0 + h * v) - J_of(u0 - h * v)) / (2 * h)
            row[f"fd_h{h:.1e}"] = fd
            row[f"rel_fp64_h{h:.1e}"] = abs(ad64 - fd) / abs(fd)
        rows.append(row)
    out["directions"] = rows
    if scales:
        h0 = scales[0] * unorm
        out["fd_rel_err_fp64_by_h"] = []
        for sc in scales:
            rel = [r[f"rel_fp64_h{sc * unorm:.1e}"] for r in rows]
            out["fd_rel_err_fp64_by_h"].append({"h_over_norm": sc, "h": sc * unorm, "max": max(rel),
                                                "median": float(np.median(rel))})
    rel = [r[f"rel_fp64_h{h0:.1e}"] for r in rows]
    out["fd_rel_err_fp64"] = {"h": h0, "max": max(rel), "median": float(np.median(rel))}
    out["fd_rel_err_fp32_adjoint"] = float(np.median(
        [abs(r["adjoint_fp32"] - r[f"fd_h{h0:.1e}"]) / abs(r[f"fd_h{h0:.1e}"]) for r in rows]))
    fsim.close()
    print(json.dumps(out), flush=True)


def config_dict():
    return {"workload": f"taylor-green-{N_GRID}^3 fp32 linear-WENO5 smooth-GKS S2O4",
            "model": "HGKS", "grid": [N_GRID] * 3, "precision": "fp32", "recon": "linear",
            "flux": "smooth", "cfl": 0.5, "mach": 0.1, "reynolds": 1600, "prandtl": 0.72,
            "global_batch": 1, "seq_len": None, "parallelism": "replicas",
            "l2": "inputs larger than L2: the FP32 state alone is 335 MB per step"}


def job_rate(seconds_local: float, cells_per_rank: int, dist=None, device: str = "cpu"):
    """Whole-job rate of independent replicas, one per rank: the slowest
    rank's time per step (max over ranks) and the cells all ranks advanced per
    second, in Mcell-updates/s.  `dist` is torch.distributed with an
    initialised process group (None for one process); `device` holds the
    reduction tensor ("cuda" for NCCL, "cpu" for gloo)."""
    world, t = 1, seconds_local
    if dist is not None:
        import torch
        world = dist.get_world_size()
        x = torch.tensor([seconds_local], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, world * cells_per_rank / t / 1e6


def run_ours(args, rank: int, world: int):
    import torch
    from paper_2005_08736_gb300 import build as cuda_build
    from paper_2005_08736_gb300 import inputs
    from paper_2005_08736_gb300.solver import Simulation, measure_fp_peaks, taylor_green_config

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        cuda_build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        dist.barrier()
        cuda_build.build()

    def barrier():
        if dist is not None:
            dist.barrier()

    prim = inputs.taylor_green(N_GRID)
    cfg = taylor_green_config(N_GRID, args.precision, args.recon, args.flux,
                              recon_vars=1 if args.char else 0)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    if args.shape:
        v, c = (int(x) for x in args.shape.split(","))
        sim._call(sim.lib.hgks_set_sweep_shape(sim.h, v, c))
        tune = {"variant": v, "chunk": c, "fixed": True}
    else:
        tune = sim.autotune()  # launch shape of the sweep kernel for this grid
    stream = sim.stream
    for _ in range(args.warmup):
        sim.step(1, sync=False)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        sim.step(args.steps, sync=False)
        stop.record(stream)
        torch.cuda.synchronize()
    barrier()
    s_step, value = job_rate(start.elapsed_time(stop) / args.steps * 1e-3, cfg.cells, dist, "cuda")
    ms = 1e3 * s_step
    t_reached = sim.step(0)  # sync + non-physical check

    # Kernel classes of one step (CUDA events around each launch).
    prof = sim.profile_step()
    if args.quick:
        sim.close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "Mcell-updates/s",
                              "ms_per_step": ms, "grid": N_GRID, "precision": args.precision,
                              "recon": args.recon, "flux": args.flux, "char": args.char,
                              "autotune": tune,
                              "kernel_ms_per_step": prof, "quick": True}), flush=True)
        return

    # FP64 step of the same workload, and the FP32-vs-FP64 error after the same steps.
    k64 = max(2, min(args.steps, 4))
    sim64 = Simulation(taylor_green_config(N_GRID, "fp64"))
    sim64.init_primitive(prim)
    sim64.step(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(sim64.stream)
    sim64.step(k64, sync=False)
    e1.record(sim64.stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / k64
    # Error of FP32 against FP64 after 1 + k64 steps from the same initial state.
    # The FP32 context takes the timed launch shape.
    simA = Simulation(taylor_green_config(N_GRID, "fp32"))
    simA._call(simA.lib.hgks_set_sweep_shape(simA.h, int(tune["variant"]), int(tune["chunk"])))
    simA.init_primitive(prim)
    simA.step(1 + k64)
    a32, a64 = simA.state(), sim64.state()
    err_var = [float(np.abs(a32[v] - a64[v]).max() / np.abs(a64[v]).max()) for v in range(5)]
    mom_scale = max(float(np.abs(a64[v]).max()) for v in (1, 2, 3))
    err_shared = max(float(np.abs(a32[v] - a64[v]).max()) / (mom_scale if v in (1, 2, 3)
                                                             else float(np.abs(a64[v]).max()))
                     for v in range(5))
    ek32, ek64 = simA.diagnostics()["Ek"], sim64.diagnostics()["Ek"]
    simA.close()
    sim64.close()
    # FP32 against the FP64 oracle itself at 32^3 (Taylor-Green, 20 CFL steps,
    # the oracle's stored state), in the same run.
    g = np.load(os.path.join(ROOT, "tests", "golden", "tg32_linear_smooth_20steps.npz"))
    s32 = Simulation(taylor_green_config(32, "fp32"))
    s32._call(s32.lib.hgks_set_sweep_shape(s32.h, int(tune["variant"]), 0))
    s32.init_primitive(inputs.taylor_green(32))
    s32.step(20)
    b32 = s32.state()
    s32.close()
    ref32 = g["state"]
    err_or32 = [float(np.abs(b32[v] - ref32[v]).max() / np.abs(ref32[v]).max()) for v in range(5)]

    # End to end through the C ABI with host buffers: per step the FP64
    # primitive state is copied in from pinned host memory, one step runs and
    # the stepped FP64 conservative state is copied back into pinned host
    # memory (hgks_get_state with a host pointer, which synchronises).
    host = torch.from_numpy(np.ascontiguousarray(prim)).pin_memory()
    host_out = torch.empty(cfg.shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.init_primitive(host)
        sim.step(1, sync=False)
        sim.state(out=host_out)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_finite = bool(torch.isfinite(host_out).all())
    barrier()
    sim.close()
    e2e_s, e2e_value = job_rate(e2e_s, cfg.cells, dist, "cuda")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = load_peaks()
    sm_clock = clocks.summary()
    faces_per_launch = (N_GRID + 1) * N_GRID * N_GRID
    flux_ms = prof["flux_stage1"] / 3.0  # average launch duration of the dominant kernel
    sms, lanes = torch.cuda.get_device_properties(local).multi_processor_count, 128
    clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    nominal_tflops = sms * lanes * 2 * clock_mhz * 1e6 / 1e12
    fp_peaks = measure_fp_peaks()  # FMA throughput of this GPU, outside the timed region
    peak_tflops = fp_peaks["fp32"]
    counts = SWEEP_COUNTS[tune["variant"]]
    alg1, alg2 = alg_flops_per_face(cfg, 1), alg_flops_per_face(cfg, 2)
    achieved = alg1["flops"] * faces_per_launch / (flux_ms * 1e-3) / 1e12
    traffic = counts["dram"] * faces_per_launch if counts["dram"] else None
    roofline = {"bound": "alu",
                "kernel": f"k_sweep stage 1 (FP32, linear WENO5, smooth flux, tile {counts['tile']})",
                "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops,
                "traffic": traffic,
                "flops_per_launch": alg1["flops"] * faces_per_launch,
                "alg_flops_per_face": alg1,
                "flops_note": "algorithmic (hgks_count_flops): the kernel's closed forms tallied on "
                              "the host per face, no halo recomputation, common subexpressions "
                              "once, dead results not counted, erf/exp/sqrt not counted",
                "executed_flops_per_launch": counts["flops"] * faces_per_launch,
                "executed_note": "ncu fadd + fmul + 2 ffma per face at 128^3 (halo recomputation and "
                                 "the polynomial work of erf/exp included)",
                "peak_source": "measured: FP32 FMA throughput of this GPU (hgks_measure_fp_peaks)",
                "nominal_peak": nominal_tflops,
                "nominal_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x {clock_mhz:.0f} MHz",
                "frac_of_nominal": achieved / nominal_tflops,
                "measured_fma_tflops": fp_peaks,
                "launch_ms": flux_ms, "kernel_ms_per_step": prof,
                "hbm_frac": (traffic / (flux_ms * 1e-3) / (peaks.get("hbm_gbs", 6802.0) * 1e9)
                             if traffic else None)}
    # The whole step against its own roofline: the slower of its algorithmic
    # FP32 work at the measured FMA peak and its algorithmic HBM bytes at the
    # measured copy bandwidth.
    step_flops = 3 * faces_per_launch * (alg1["flops"] + alg2["flops"])
    step_bytes = ALG_BYTES_PER_CELL_STEP * cfg.cells
    t_alu = step_flops / (peak_tflops * 1e12) * 1e3
    t_hbm = step_bytes / (peaks.get("hbm_gbs", 6802.0) * 1e9) * 1e3
    step_roofline = {"flops_per_step": step_flops, "bytes_per_step": step_bytes,
                     "alu_bound_ms": t_alu, "hbm_bound_ms": t_hbm,
                     "bound": "alu" if t_alu >= t_hbm else "hbm",
                     "frac": max(t_alu, t_hbm) / ms,
                     "note": "algorithmic flops of the six sweeps (halo excluded) at the measured "
                             "FP32 FMA peak vs 120 B per cell-step at the measured HBM copy rate"}
    cpu_rate, cpu_s, cpu_steps = oracle_sample(1, 32, seconds=10.0)
    cpu_cores = oracle_threads()
    cpu1_rate, cpu1_s = oracle_sample_one_core()
    extras = extra_workloads(min(args.steps, 10), peak_tflops) if not args.no_extras else None
    line = {
        "metric": METRIC, "value": value, "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_MCUPS_256, "dtype": "f32", "data": "synthetic",
        "config": config_dict(),
        "fp64": {"value": world * cfg.cells / (ms64 * 1e-3) / 1e6, "unit": "Mcell-updates/s",
                 "ms_per_step": ms64, "steps": k64},
        "fp32_speedup_over_fp64": ms64 / ms,
        "fp32_error": {
            "reference": f"the FP64 GPU path at {N_GRID}^3 (itself checked against the FP64 oracle "
                         "to 1e-12 at 32^3 and on sampled cells at 256^3)",
            "steps": 1 + k64,
            "rel_linf_shared_momentum": err_shared,
            "rel_linf_per_variable": err_var,
            "metric": "max over variables of max|FP32 - FP64| / max|FP64| of the variable; "
                      "rel_linf_shared_momentum measures the three momentum components against "
                      "the largest momentum magnitude (rho W of Taylor-Green starts at zero)",
            "Ek_rel_diff": abs(ek32 - ek64) / ek64,
            "vs_oracle_32": {"steps": 20, "rel_linf_per_variable": err_or32,
                             "rel_linf": max(err_or32),
                             "reference": "FP64 oracle (tests/golden/tg32_linear_smooth_20steps.npz)"}},
        "t_reached": t_reached,
        "roofline": roofline,
        "step_roofline": step_roofline,
        "cpu_baseline": {"value": cpu_rate, "unit": "Mcell-updates/s", "cores": cpu_cores,
                         "kind": "oracle",
                         "sample": f"FP64 CPU oracle, {cpu_steps} steps of Taylor-Green 32^3 "
                                   f"({cpu_s:.1f} s), same physics and scheme",
                         "one_core": {"value": cpu1_rate, "cores": 1,
                                      "sample": f"1 step of Taylor-Green 32^3 ({cpu1_s:.1f} s)"}},
        "e2e": {"value": e2e_value, "unit": "Mcell-updates/s",
                "h2d_bytes_per_step": int(prim.nbytes), "d2h_bytes_per_step": int(host_out.numel() * 8),
                "note": "per step: FP64 primitive state host->device (pinned), one S2O4 step, FP64 "
                        "conservative state device->host (pinned)",
                "state_finite": e2e_finite},
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "clocks": sm_clock,
        "workloads": extras,
        "autotune": tune,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=256, help="grid size (profiling cases)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--recon", default="linear", choices=["linear", "weno-js", "weno-z"],
                    help="reconstruction (profiling cases; the headline uses linear)")
    ap.add_argument("--flux", default="smooth", choices=["smooth", "full"],
                    help="flux (profiling cases; the headline uses smooth)")
    ap.add_argument("--char", action="store_true",
                    help="WENO in characteristic variables (profiling cases)")
    ap.add_argument("--shape", default="",
                    help="V,C: sweep tile variant and march length (skips the autotuner)")
    ap.add_argument("--history", action="store_true",
                    help="Taylor-Green E_k / dissipation history, FP32 against FP64")
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--t-end-fp64", type=float, default=None,
                    help="--history: end time of the FP64 run (default: --t-end)")
    ap.add_argument("--errors", action="store_true",
                    help="FP32 against FP64 on the isotropic and channel workloads")
    ap.add_argument("--tau-num", type=float, default=None,
                    help="--gradcheck: C of the numerical collision time (default 1)")
    ap.add_argument("--gradcheck", action="store_true",
                    help="adjoint gradient of E_k(50) at 64^3 against central differences")
    ap.add_argument("--fd-scales", default="",
                    help="--gradcheck: comma-separated step sizes h / |u0| of the differences")
    ap.add_argument("--adjoint", action="store_true",
                    help="adjoint / forward step time at 64^3 (full and smooth flux, FP32 and FP64)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the isotropic, channel, adjoint and ensemble measurements")
    ap.add_argument("--quick", action="store_true",
                    help="time the step only (no FP64 leg, e2e or CPU baseline); for profiling")
    args = ap.parse_args()
    args.grid_given = "--grid" in sys.argv
    global N_GRID
    N_GRID = args.grid
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gradcheck:
        run_gradcheck(args)
    elif args.adjoint:
        run_adjoint(args)
    elif args.history:
        run_history(args)
    elif args.errors:
        run_errors(args)
    elif args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
