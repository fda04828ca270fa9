"""Parity of the device turbulence statistics (hgks_turbulence_stats) with the
oracle's (oracle/turbulence.py) on the same state, and their closed forms at
full size (Sec. 3.1, Sec. 3.4)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.turbulence import KEYS, statistics  # noqa: E402
from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300._lib import HGKS_E_UNSUPPORTED, HgksError  # noqa: E402
from paper_2005_08736_gb300.solver import Config, Simulation, taylor_green_config  # noqa: E402

TOL = 1e-11


def iso_config(n, prec, k0=4.0):
    c = inputs.isotropic_constants(k0=k0, mach_t=0.5)
    return Config(n, n, n, prec=prec, recon=2, flux=1, tau_num_C=1.0, prandtl=0.7, visc=1,
                  mu_ref=c["mu0"], T_ref=c["T0"], visc_exp=0.76, p_ref=c["p0"], rho_ref=1.0)


def oracle_stats(cfg: Config, cons):
    return statistics(cons, lengths=(cfg.lx, cfg.ly, cfg.lz), gamma=cfg.gamma, rho0=cfg.rho_ref,
                      visc_law=cfg.visc, mu_ref=cfg.mu_ref, T_ref=cfg.T_ref, visc_exp=cfg.visc_exp)


def compare(gpu: dict, ref: dict, tol: float):
    # Scale of each entry: its own magnitude, or for quantities that may
    # vanish by symmetry the magnitude of a related non-vanishing one.
    scale = {"Su": 1.0, "Fu": 1.0, "eps2": ref["eps1"], "eps3": abs(ref["p_theta"]) + ref["eps1"],
             "p_theta": abs(ref["p_theta"]) + ref["eps1"], "eps_d": ref["eps_s"],
             "theta_rms": ref["omega_rms"]}
    for a in "xyz":
        m2 = ref[f"du2_{a}"]
        scale[f"du3_{a}"] = m2 ** 1.5
        scale[f"du4_{a}"] = m2 * m2
    bad = {}
    for k in KEYS:
        s = max(abs(ref[k]), scale.get(k, 0.0), 1e-300)
        e = abs(gpu[k] - ref[k]) / s
        if e > tol:
            bad[k] = (gpu[k], ref[k], e)
    assert not bad, bad


@pytest.mark.parametrize("prec", [0, 1])
def test_isotropic_statistics_match_oracle(prec):
    cfg = iso_config(32, prec)
    sim = Simulation(cfg)
    sim.init_primitive(inputs.isotropic(32, 0, k0=4.0))
    sim.step(5)
    gpu = sim.turbulence()
    ref = oracle_stats(cfg, sim.state())
    sim.close()
    compare(gpu, ref, TOL)
    assert gpu["rho_rms"] > 0 and gpu["eps_d"] > 0 and gpu["Fu"] > 1.0


def test_ragged_grid_statistics_match_oracle():
    cfg = Config(20, 13, 11, lx=3.0, ly=2.0, lz=1.7, prec=0, visc=1, mu_ref=0.01, T_ref=1.0,
                 visc_exp=0.76, p_ref=1.0, rho_ref=1.0)
    prim = inputs.random_smooth((20, 13, 11), seed=5, amp=0.2, kmax=2)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    gpu = sim.turbulence()
    ref = oracle_stats(cfg, sim.state())
    sim.close()
    compare(gpu, ref, TOL)


def test_taylor_green_256_closed_forms():
    """Full size, in the benchmark's precision: the initial enstrophy is
    3/8 g^2 (g the sixth-order difference symbol of sin x), theta vanishes,
    and after steps the summation-by-parts identity rho0 eps1 = eps_s + eps_d
    of periodic grids holds (constant mu)."""
    n = 256
    cfg = taylor_green_config(n, "fp32")
    sim = Simulation(cfg)
    sim.init_primitive(inputs.taylor_green(n))
    s0 = sim.turbulence()
    h = 2 * math.pi / n
    g = (45 * math.sin(h) - 9 * math.sin(2 * h) + math.sin(3 * h)) / (30 * h)
    # FP32 storage of the velocity: ~1e-7 relative
    assert s0["zeta"] == pytest.approx(0.375 * g * g, rel=1e-6)
    assert s0["Ek"] == pytest.approx(0.125, rel=1e-6)
    assert s0["theta_rms"] < 1e-5 * s0["omega_rms"]
    assert s0["Fu"] == pytest.approx(27.0 / 8.0, rel=1e-5)
    sim.step(4)
    s1 = sim.turbulence()
    sim.close()
    assert cfg.rho_ref * s1["eps1"] == pytest.approx(s1["eps_s"] + s1["eps_d"], rel=1e-10)
    assert 0 < s1["Ek"] < s0["Ek"]


def test_rejects_walls():
    cfg = Config(16, 16, 16, ly=2.0, y0=-1.0, y_stretch=1, stretch_b=2.0, bc_y=1,
                 T_wall=100 / 1.4, prec=0)
    sim = Simulation(cfg)
    sim.init_primitive(inputs.channel(16, 16, 16, 0))
    with pytest.raises(HgksError) as ei:
        sim.turbulence()
    sim.close()
    assert ei.value.status == HGKS_E_UNSUPPORTED


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_history_matches_the_oracle_run(prec):
    """The device statistics history (hgks_history_start / _read) of a
    Taylor-Green run with CFL steps (uneven times): every record against
    the oracle's statistics of the oracle's state at the same step, and
    eps(E_k), eps_num against the oracle's second-order differences
    (Sec. 3.1).  FP32: the records at the FP32 state tolerance (the
    differences of FP32 E_k samples are not compared)."""
    import oracle
    from oracle.turbulence import dissipation_history
    n, every, steps = 24, 2, 10
    cfg = taylor_green_config(n, prec)
    cfg64 = taylor_green_config(n, "fp64")
    prim = inputs.taylor_green(n)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    sim.history_start(every, capacity=5)   # steps 0, 2, 4, 6, 8 fit; step 10 is dropped
    sim.step(steps)
    recs = sim.history()
    sim.history_stop()
    sim.step(2)
    assert len(sim.history()) == 5         # no recording after the stop
    sim.close()
    o = oracle.Solver(oracle.Config(n, n, n, recon=0, flux=0, prandtl=cfg.prandtl, mu_ref=cfg.mu_ref,
                                    cfl=cfg.cfl))
    o.set_state(oracle.conservative(prim, 1.4))
    times, stats = [], []
    for k in range(0, 9, every):
        if k:
            o.step(every)
        times.append(o.t)
        stats.append(oracle_stats(cfg64, o.state()))
    eps_ek, eps_num = dissipation_history(times, stats)
    assert [r["step"] for r in recs] == [0, 2, 4, 6, 8]
    tol = TOL if prec == "fp64" else 2e-5
    for r, t, ref, e, en in zip(recs, times, stats, eps_ek, eps_num):
        assert r["t"] == pytest.approx(t, rel=1e-13 if prec == "fp64" else 1e-6, abs=1e-300)
        compare(r, ref, tol)
        if prec == "fp64":
            assert r["eps_Ek"] == pytest.approx(e, rel=1e-6)
            assert abs(r["eps_num"] - en) <= 1e-6 * abs(e)
