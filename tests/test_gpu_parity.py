"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

* Taylor-Green 32^3, 20 CFL-0.5 steps, FP64, both scheme modes, against the
  oracle's stored states (tests/golden/make_oracle_goldens.py): relative
  L-infinity <= 1e-12 per variable.
* Ragged small grids (several tiles and a ragged tail) in every
  reconstruction / flux mode, and the stretched wall-bounded channel with the
  body force, against the live oracle.
* The full-size 256^3 Taylor-Green step in the launch configuration of the
  benchmark, on sampled cells: the oracle steps a 15^3 periodic patch around
  each sampled cell (the cell's one-step result depends only on cells within
  6 of it).
* FP32 against the oracle within a tolerance derived from the arithmetic (below).
* Properties: free-stream preservation, conservation, graph replay, the
  non-physical-state report.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300._lib import HGKS_E_INVAL, HGKS_E_NONPHYSICAL, HgksError  # noqa: E402
from paper_2005_08736_gb300.solver import Config, Simulation, taylor_green_config  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FP64_TOL = 1e-12
# FP32 bound on the per-variable relative L-infinity error against the FP64
# oracle: one FP32 step rounds each flux to ~6e-8 relative, the divergence of
# the enthalpy flux h_r U (h_r = 250 at Ma 0.1) amplifies it by h_r/|d(rho E)| ~ 1e2,
# and 20 steps accumulate ~sqrt(20) of that.
FP32_TOL = 2e-5

MODES = [("linear", "smooth"), ("weno-js", "full"), ("weno-z", "full"), ("weno-z", "smooth"),
         ("linear", "full")]
ORACLE_RECON = {"linear": 0, "weno-js": 1, "weno-z": 2}
ORACLE_FLUX = {"smooth": 0, "full": 1}


def rel_linf(a, b):
    """max over variables of max|a_v - b_v| / max|b_v|."""
    a, b = np.asarray(a), np.asarray(b)
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def oracle_cfg(c: Config) -> oracle.Config:
    return oracle.Config(c.nx, c.ny, c.nz, lx=c.lx, ly=c.ly, lz=c.lz, x0=c.x0, y0=c.y0, z0=c.z0,
                         y_stretch=c.y_stretch, stretch_b=c.stretch_b, bc_y=c.bc_y, gamma=c.gamma,
                         prandtl=c.prandtl, visc_law=c.visc, mu_ref=c.mu_ref, T_ref=c.T_ref,
                         visc_exp=c.visc_exp, T_wall=c.T_wall, force_x=c.force_x, recon=c.recon,
                         flux=c.flux, tau_num_C=c.tau_num_C, cfl=c.cfl,
                         force_mode=c.force_mode, mass_flux=c.mass_flux,
                         char_recon=c.recon_vars)


def run_both(cfg: Config, prim, steps, dt=0.0):
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    t = sim.step(steps, dt)
    gpu = sim.state()
    sim.close()
    o = oracle.Solver(oracle_cfg(cfg))
    o.set_state(oracle.conservative(prim, cfg.gamma))
    o.step(steps, dt)
    return gpu, o.state(), t, o.t


@pytest.mark.parametrize("recon,flux,name", [("linear", "smooth", "linear_smooth"),
                                             ("weno-z", "full", "wenoz_full")])
def test_taylor_green_32_fp64_matches_oracle_after_20_steps(recon, flux, name):
    ref = np.load(os.path.join(GOLDEN, f"tg32_{name}_20steps.npz"))
    cfg = taylor_green_config(32, "fp64", recon, flux)
    sim = Simulation(cfg)
    sim.init_primitive(inputs.taylor_green(32))
    t = sim.step(20)
    err = rel_linf(sim.state(), ref["state"])
    assert t == pytest.approx(float(ref["t"]), rel=1e-13)
    assert err <= FP64_TOL, err


@pytest.mark.parametrize("recon,flux", MODES)
def test_ragged_grid_fp64_matches_oracle(recon, flux):
    n = (13, 10, 9)
    cfg = Config(*n, prec=0, recon=ORACLE_RECON[recon], flux=ORACLE_FLUX[flux], tau_num_C=1.0,
                 mu_ref=5e-3, p_ref=1.0, prandtl=0.7, visc=1, T_ref=1.0, visc_exp=0.76)
    prim = inputs.random_smooth(n, seed=5, amp=0.15)
    gpu, ref, t, to = run_both(cfg, prim, 3)
    assert t == pytest.approx(to, rel=1e-13)
    assert rel_linf(gpu, ref) <= FP64_TOL


@pytest.mark.parametrize("recon,flux", [("weno-js", "smooth"), ("weno-z", "smooth"),
                                        ("weno-js", "full"), ("weno-z", "full"), ("linear", "full")])
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_characteristic_reconstruction_matches_oracle(recon, flux, prec, tol):
    """WENO in characteristic variables (Sec. 2.1, Remark 1) on a ragged grid
    (several tiles and a ragged tail); with linear weights the projection is
    skipped on the device and the oracle's projected result must agree."""
    n = (13, 10, 9)
    cfg = Config(*n, prec=prec, recon=ORACLE_RECON[recon], flux=ORACLE_FLUX[flux], tau_num_C=1.0,
                 mu_ref=5e-3, p_ref=1.0, prandtl=0.7, visc=1, T_ref=1.0, visc_exp=0.76,
                 recon_vars=1)
    prim = inputs.random_smooth(n, seed=8, amp=0.3)
    gpu, ref, t, to = run_both(cfg, prim, 3)
    assert t == pytest.approx(to, rel=1e-13 if prec == 0 else 1e-6)
    assert rel_linf(gpu, ref) <= tol


def channel_cfg(nx, ny, nz, prec):
    return Config(nx, ny, nz, lx=2 * math.pi, ly=2.0, y0=-1.0, lz=math.pi, y_stretch=1,
                  stretch_b=2.0, bc_y=1, T_wall=100 / 1.4, mu_ref=0.0541 / 180, force_x=2.93e-3,
                  prec=prec, recon=0, flux=0)


def channel_prim(nx, ny, nz, seed=0):
    yf = inputs.channel_faces(ny)
    yc = 0.5 * (yf[1:] + yf[:-1])
    rng = np.random.Generator(np.random.PCG64(seed))
    U = 1.5 * (1 - yc ** 2)[None, :, None] * np.ones((nz, ny, nx))
    prim = np.zeros((5, nz, ny, nx))
    prim[0] = 1.0
    prim[1] = U * (1 + 0.1 * rng.uniform(-1, 1, U.shape))
    prim[2] = 0.1 * U * rng.uniform(-1, 1, U.shape)
    prim[3] = 0.1 * U * rng.uniform(-1, 1, U.shape)
    prim[4] = 100 / 1.4
    return prim


def test_channel_with_walls_fp64_matches_oracle():
    cfg = channel_cfg(12, 16, 10, prec=0)
    gpu, ref, t, to = run_both(cfg, channel_prim(12, 16, 10), 3)
    assert t == pytest.approx(to, rel=1e-13)
    assert rel_linf(gpu, ref) <= FP64_TOL


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_channel_constant_mass_flux_matches_oracle(prec, tol):
    """Sec. 3.3 after transition: the force keeps the volume integral of rho U
    at its target; the device force of every step matches the oracle's."""
    n = (12, 16, 10)
    cfg = channel_cfg(*n, prec=prec)
    cfg.force_mode, cfg.mass_flux = 1, 1.02
    prim = channel_prim(*n)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    o = oracle.Solver(oracle_cfg(cfg))
    o.set_state(oracle.conservative(prim, cfg.gamma))
    for _ in range(3):
        sim.step(1)
        o.step(1)
        d = sim.diagnostics()
        # f_x dt is the correction of <rho U> ~ 1 (per unit density), formed
        # from a difference of O(1) totals: its error is the state tolerance.
        assert abs(d["force_x"] - o.last_force) * d["dt"] <= 10 * tol * cfg.mass_flux
    gpu = sim.state()
    d = sim.diagnostics()
    sim.close()
    assert rel_linf(gpu, o.state()) <= tol
    vol = cfg.lx * cfg.ly * cfg.lz
    assert d["mom"][0] / vol == pytest.approx(1.02, rel=1e-12 if prec == 0 else 1e-6)


@pytest.mark.parametrize("variant", [1, 3])
def test_channel_fp32_tile_variants_match_oracle(variant):
    """The wider and the packed sweep tiles with walls, the stretched y grid and
    the body force (FP32, ragged 40 x 24 x 18 grid: several tiles and a ragged
    tail in every direction)."""
    n = (40, 24, 18)
    cfg = channel_cfg(*n, prec=1)
    prim = channel_prim(*n)
    sim = Simulation(cfg)
    sim._call(sim.lib.hgks_set_sweep_shape(sim.h, variant, 0))
    sim.init_primitive(prim)
    sim.step(3)
    gpu = sim.state()
    sim.close()
    o = oracle.Solver(oracle_cfg(cfg))
    o.set_state(oracle.conservative(prim, cfg.gamma))
    o.step(3)
    err = rel_linf(gpu, o.state())
    print(f"channel FP32 variant {variant}: relative L-inf error against the oracle {err:.3e}")
    assert err <= FP32_TOL, err


def test_minimum_grid_and_fixed_dt():
    cfg = taylor_green_config(6, "fp64", "weno-z", "full")
    gpu, ref, t, to = run_both(cfg, inputs.taylor_green(6), 2, dt=0.01)
    assert t == pytest.approx(0.02, rel=1e-14)
    assert rel_linf(gpu, ref) <= FP64_TOL


def patch_step(prim_full, centre, dt, cfg: Config, R=7, steps=1):
    """Oracle steps of the (2R+1)^3 periodic patch around `centre` (x, y, z);
    a cell's result after k steps depends on cells within 6k of it."""
    assert R >= 6 * steps + 1
    nz, ny, nx = prim_full.shape[1:]
    ix = (np.arange(-R, R + 1) + centre[0]) % nx
    iy = (np.arange(-R, R + 1) + centre[1]) % ny
    iz = (np.arange(-R, R + 1) + centre[2]) % nz
    patch = prim_full[:, iz][:, :, iy][:, :, :, ix]
    m = 2 * R + 1
    oc = oracle_cfg(cfg)
    oc.nx = oc.ny = oc.nz = m
    oc.lx, oc.ly, oc.lz = cfg.lx / nx * m, cfg.ly / ny * m, cfg.lz / nz * m
    o = oracle.Solver(oc)
    o.set_state(oracle.conservative(patch, cfg.gamma))
    o.step(steps, dt)
    return o.state()[:, R, R, R]


SAMPLES = [(0, 0, 0), (255, 17, 128), (64, 200, 31), (130, 129, 254), (32, 96, 160),
           (200, 250, 7), (127, 0, 64), (90, 45, 222)]


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_full_size_256_steps_on_sampled_cells(prec, tol):
    """Two steps of the 256^3 benchmark workload in its timed launch shape,
    on 8 sampled cells: the oracle steps the 27^3 periodic patch around each
    (two steps reach 12 cells).  Metric: per variable, the momentum components
    measured against the largest momentum magnitude (rho W = 0 at the start;
    the FP32 error statement of this library uses the same metric)."""
    n, dt, steps = 256, 1.1e-3, 2
    cfg = taylor_green_config(n, prec)
    prim = inputs.taylor_green(n)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    sim.autotune()  # the launch shape bench.py times
    sim.init_primitive(prim)
    sim.step(steps, dt)
    gpu = sim.state()
    sim.close()
    Q0 = oracle.conservative(prim, 1.4)
    scale = np.abs(Q0).reshape(5, -1).max(axis=1)
    scale[1:4] = scale[1:4].max()  # momentum components share one scale (rho W = 0 here)
    for c in SAMPLES:
        ref = patch_step(prim, c, dt, cfg, R=13, steps=steps)
        got = gpu[:, c[2], c[1], c[0]]
        err = (np.abs(got - ref) / scale).max()
        assert err <= tol, (c, err)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_fp32_taylor_green_32_error_against_oracle(variant):
    # every sweep tile variant of the linear-weight smooth FP32 step, the
    # packed one (3) included
    ref = np.load(os.path.join(GOLDEN, "tg32_linear_smooth_20steps.npz"))
    cfg = taylor_green_config(32, "fp32")
    sim = Simulation(cfg)
    sim._call(sim.lib.hgks_set_sweep_shape(sim.h, variant, 0))
    sim.init_primitive(inputs.taylor_green(32))
    sim.step(20)
    err = rel_linf(sim.state(), ref["state"])
    print(f"FP32 TG 32^3 20 steps, variant {variant}: relative L-inf error against the FP64 "
          f"oracle = {err:.3e}")
    assert err <= FP32_TOL, err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_free_stream_is_preserved(prec):
    n = (9, 8, 7)
    prim = np.zeros((5, 7, 8, 9))
    prim[0], prim[1], prim[2], prim[3], prim[4] = 1.0, 0.3, -0.2, 0.1, 100 / 1.4
    for recon, flux in (("linear", "smooth"), ("weno-z", "full")):
        cfg = Config(*n, prec=0 if prec == "fp64" else 1, recon=ORACLE_RECON[recon],
                     flux=ORACLE_FLUX[flux], tau_num_C=1.0)
        sim = Simulation(cfg)
        sim.init_primitive(prim)
        before = sim.state()
        sim.step(3)
        assert np.array_equal(sim.state(), before)


def test_periodic_totals_conserved_fp64():
    n = (24, 20, 16)
    cfg = Config(*n, prec=0, recon=2, flux=1, tau_num_C=1.0, mu_ref=1e-3, p_ref=1.0)
    sim = Simulation(cfg)
    sim.init_primitive(inputs.random_smooth(n, seed=9, amp=0.2))
    d0 = sim.diagnostics()
    sim.step(5)
    d1 = sim.diagnostics()
    for k in ("mass", "energy"):
        assert abs(d1[k] - d0[k]) <= 1e-13 * abs(d0[k])
    for a, b in zip(d1["mom"], d0["mom"]):
        assert abs(a - b) <= 1e-13 * d0["mass"]


def test_graph_replay_equals_single_steps():
    cfg = taylor_green_config(16, "fp32")
    a, b = Simulation(cfg), Simulation(cfg)
    prim = inputs.taylor_green(16)
    a.init_primitive(prim)
    b.init_primitive(prim)
    a.step(4)
    for _ in range(4):
        b.step(1)
    assert np.array_equal(a.state(), b.state())


def test_zero_steps_leave_state_and_time_unchanged():
    # The empty call: no step runs, the state check still runs; a negative
    # count is rejected before any device work.
    for prec in ("fp64", "fp32"):
        sim = Simulation(taylor_green_config(8, prec))
        sim.init_primitive(inputs.taylor_green(8))
        q0 = sim.state()
        assert sim.step(0) == 0.0
        assert np.array_equal(sim.state(), q0)
        with pytest.raises(HgksError) as e:
            sim.step(-1)
        assert e.value.status == HGKS_E_INVAL
        sim.close()


def test_nonphysical_state_is_reported():
    cfg = taylor_green_config(8, "fp64")
    prim = inputs.taylor_green(8)
    prim[4, 2, 3, 4] = -1.0  # negative pressure planted on the host
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    with pytest.raises(HgksError) as e:
        sim.step(1)
    assert e.value.status == HGKS_E_NONPHYSICAL


def separating_flow():
    """u = +4 in the middle half of x, -4 outside (rho = p = 1): two
    rarefactions so strong that the WENO-Z / full-flux step with dt = 0.01
    is non-physical at step 3 (the oracle: rho_min 0.80 after step 2, NaN
    after step 3)."""
    prim = np.zeros((5, 8, 8, 16))
    prim[0], prim[4] = 1.0, 1.0
    x = (np.arange(16) + 0.5) / 16 * 2 * math.pi
    prim[1] = np.where((x > math.pi / 2) & (x < 1.5 * math.pi), 4.0, -4.0)[None, None, :]
    return prim


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonphysical_step_leaves_the_last_good_state(prec):
    """E_NONPHYSICAL leaves the state, time and step count at the last good
    step, whether the steps ran one per call or in one batch of graph
    replays; stepping can resume afterwards."""
    cfg = Config(16, 8, 8, prec=0 if prec == "fp64" else 1, recon=2, flux=1, tau_num_C=1.0,
                 mu_ref=1e-3, p_ref=1.0)
    prim, dt = separating_flow(), 0.01
    one = Simulation(cfg)
    one.init_primitive(prim)
    failed = None
    for k in range(1, 7):
        try:
            one.step(1, dt)
        except HgksError as e:
            assert e.status == HGKS_E_NONPHYSICAL
            failed = k
            break
    assert failed is not None and failed >= 2, failed
    good = Simulation(cfg)
    good.init_primitive(prim)
    good.step(failed - 1, dt)
    ref, dref = good.state(), good.diagnostics()
    assert dref["rho_min"] > 0 and dref["p_min"] > 0
    batch = Simulation(cfg)
    batch.init_primitive(prim)
    with pytest.raises(HgksError) as e:
        batch.step(6, dt)
    assert e.value.status == HGKS_E_NONPHYSICAL
    for sim in (one, batch):
        d = sim.diagnostics()
        assert np.array_equal(sim.state(), ref)
        assert d["step"] == failed - 1 and d["t"] == pytest.approx(dref["t"], rel=1e-14)
    # the flag is cleared: a smaller step from the last good state runs
    batch.step(1, dt / 100)
    assert batch.diagnostics()["step"] == failed
    for sim in (one, good, batch):
        sim.close()


def test_state_round_trip_fp64():
    cfg = taylor_green_config(10, "fp64")
    Q = oracle.conservative(inputs.taylor_green(10), 1.4)
    sim = Simulation(cfg)
    sim.init_conservative(Q)
    assert np.allclose(sim.state(), Q, rtol=0, atol=1e-13)
    dev = sim.state(device=True)
    assert np.allclose(dev.cpu().numpy(), Q, rtol=0, atol=1e-13)
