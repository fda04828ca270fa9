"""Parity of the CUDA path with the FP64 oracle on the method's edge cases.

* hgks_diagnostics (FP64 totals, E_k, rho_min, p_min) against the same sums
  formed from the oracle's state, on a periodic and on the stretched, walled
  channel grid (volume weights from the oracle's own widths).
* Data where WENO5's nonlinear weights are far from the linear ones: density
  and pressure jumps, and a double shear layer thinner than a cell, in every
  reconstruction / flux mode, conservative and characteristic variables.
* mu = 0: the collision time vanishes (tau = 0, or the numerical term alone
  with the full flux), where exp(-dt/tau) underflows to zero.
* The isotropic start of Sec. 3.4 at 32^3 (kappa0 = 4, Ma_t 0.5 and 1.0):
  power-law viscosity, WENO-Z, the full flux and the numerical collision time.
* Members of a mixed-size, mixed-mode ensemble against the oracle.

FP64 is held to 1e-12 relative L-infinity per variable.  FP32 is held to
FP32_TOL with the metric used for every FP32 error statement of this
library: per variable, max|a - b| over the scale of that variable, where the
three momentum components share one scale (the largest momentum component),
because they are the components of one vector and a component that starts at
zero (rho W of Taylor-Green) has no scale of its own.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300.solver import Config, Ensemble, Simulation  # noqa: E402

FP64_TOL = 1e-12
FP32_TOL = 2e-5

MODES = [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1), (0, 1)]  # (recon, flux)


def rel_linf(a, b):
    """max over variables of max|a_v - b_v| / max|b_v| (strict, per variable)."""
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def rel_linf_shared(a, b):
    """The FP32 error metric: per variable, the momentum components over the
    largest momentum magnitude of b."""
    scale = [max(np.abs(b[v]).max(), 1e-300) for v in range(5)]
    m = max(scale[1:4])
    scale[1:4] = [m, m, m]
    return max(np.abs(a[v] - b[v]).max() / scale[v] for v in range(5))


def oracle_cfg(c: Config) -> oracle.Config:
    return oracle.Config(c.nx, c.ny, c.nz, lx=c.lx, ly=c.ly, lz=c.lz, x0=c.x0, y0=c.y0, z0=c.z0,
                         y_stretch=c.y_stretch, stretch_b=c.stretch_b, bc_y=c.bc_y, gamma=c.gamma,
                         prandtl=c.prandtl, visc_law=c.visc, mu_ref=c.mu_ref, T_ref=c.T_ref,
                         visc_exp=c.visc_exp, T_wall=c.T_wall, force_x=c.force_x, recon=c.recon,
                         flux=c.flux, tau_num_C=c.tau_num_C, cfl=c.cfl,
                         force_mode=c.force_mode, mass_flux=c.mass_flux,
                         char_recon=c.recon_vars)


_ORACLE_CACHE = {}


def oracle_run(cfg: Config, prim, steps, dt=0.0, key=None):
    """The oracle's state and time after `steps` steps (cached by key: the
    FP64 and FP32 cases of one input share one oracle run)."""
    if key is not None and key in _ORACLE_CACHE:
        return _ORACLE_CACHE[key]
    o = oracle.Solver(oracle_cfg(cfg))
    o.set_state(oracle.conservative(prim, cfg.gamma))
    o.step(steps, dt)
    res = (o.state(), o.t, o)
    if key is not None:
        _ORACLE_CACHE[key] = res
    return res


def gpu_run(cfg: Config, prim, steps, dt=0.0):
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    t = sim.step(steps, dt)
    out = sim.state()
    sim.close()
    return out, t


# ------------------------------------------------------------- diagnostics ---

def diag_from_oracle(o: "oracle.Solver", cfg: Config) -> dict:
    """The quantities of hgks_diag formed from the oracle's state: totals
    sum Q |Omega_c|, E_k = sum rho |U|^2/2 |Omega_c| / (rho_ref |Omega|), and
    the minima of rho and p = (gamma - 1)(rho E - rho |U|^2 / 2)."""
    Q = o.state()
    wx, wy, wz = (o.widths(d) for d in range(3))
    vol = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    rho = Q[0]
    ke = 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / rho
    p = (cfg.gamma - 1.0) * (Q[4] - ke)
    return {"mass": (rho * vol).sum(), "mom": tuple((Q[k] * vol).sum() for k in (1, 2, 3)),
            "energy": (Q[4] * vol).sum(),
            "Ek": (ke * vol).sum() / (cfg.rho_ref * cfg.lx * cfg.ly * cfg.lz),
            "rho_min": rho.min(), "p_min": p.min(), "volume": vol.sum()}


def channel_cfg(nx, ny, nz, prec):
    return Config(nx, ny, nz, lx=2 * math.pi, ly=2.0, y0=-1.0, lz=math.pi, y_stretch=1,
                  stretch_b=2.0, bc_y=1, T_wall=100 / 1.4, mu_ref=0.0541 / 180, force_x=2.93e-3,
                  prec=prec, recon=0, flux=0)


@pytest.mark.parametrize("case", ["periodic", "channel"])
def test_diagnostics_match_sums_over_the_oracle_state(case):
    if case == "periodic":
        n = (14, 11, 9)
        cfg = Config(*n, prec=0, recon=2, flux=1, tau_num_C=1.0, mu_ref=2e-3, p_ref=1.0)
        prim = inputs.random_smooth(n, seed=21, amp=0.2)
    else:
        n = (12, 16, 10)
        cfg = channel_cfg(*n, prec=0)
        prim = inputs.channel(*n, seed=3)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    sim.step(3)
    d = sim.diagnostics()
    sim.close()
    _, t_o, o = oracle_run(cfg, prim, 3)
    ref = diag_from_oracle(o, cfg)
    assert d["t"] == pytest.approx(t_o, rel=1e-13)
    assert d["step"] == 3
    for k in ("mass", "energy", "Ek", "rho_min", "p_min"):
        assert abs(d[k] - ref[k]) <= FP64_TOL * abs(ref[k]), (k, d[k], ref[k])
    # momentum totals may vanish: measured against the mass scale times the
    # largest speed of the state
    mscale = ref["mass"] * max(np.abs(prim[1:4]).max(), 1e-3)
    for a, b in zip(d["mom"], ref["mom"]):
        assert abs(a - b) <= FP64_TOL * mscale, (a, b)


def test_diagnostics_fp32_within_tolerance():
    # FP32 storage, FP64 reductions: the totals carry the state's FP32 error
    n = (14, 11, 9)
    cfg = Config(*n, prec=1, recon=0, flux=0, mu_ref=2e-3, p_ref=1.0)
    prim = inputs.random_smooth(n, seed=22, amp=0.2)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    sim.step(3)
    d = sim.diagnostics()
    sim.close()
    cfg64 = Config(*n, prec=0, recon=0, flux=0, mu_ref=2e-3, p_ref=1.0)
    _, _, o = oracle_run(cfg64, prim, 3)
    ref = diag_from_oracle(o, cfg64)
    for k in ("mass", "energy", "Ek", "rho_min", "p_min"):
        assert abs(d[k] - ref[k]) <= FP32_TOL * abs(ref[k]), (k, d[k], ref[k])


# ------------------------------------------------------------ rough inputs ---

ROUGH = {
    "slab": lambda n: inputs.slab(n, seed=31, axis=1),
    "slab_z": lambda n: inputs.slab(n, seed=32, axis=2, rho=(1.0, 0.3), p=(0.5, 1.0)),
    "shear": lambda n: inputs.shear_layer(n, seed=33),
}


def rough_cfg(n, recon, flux, prec, char=0, mu=2e-3):
    return Config(*n, prec=prec, recon=recon, flux=flux, tau_num_C=1.0 if flux == 1 else 0.0,
                  mu_ref=mu, p_ref=1.0, prandtl=0.7, visc=1, T_ref=1.0, visc_exp=0.76,
                  recon_vars=char)


@pytest.mark.parametrize("field", sorted(ROUGH))
@pytest.mark.parametrize("recon,flux", MODES)
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_rough_fields_match_oracle(field, recon, flux, prec, tol):
    """Jumps and a thin shear layer on a ragged grid (several tiles and a
    ragged tail in every direction), 3 CFL steps."""
    n = (13, 17, 11)
    prim = ROUGH[field](n)
    cfg = rough_cfg(n, recon, flux, prec)
    ref, t_o, _ = oracle_run(rough_cfg(n, recon, flux, 0), prim, 3, key=("rough", field, recon, flux))
    got, t = gpu_run(cfg, prim, 3)
    assert t == pytest.approx(t_o, rel=1e-13 if prec == 0 else 1e-6)
    err = rel_linf(got, ref) if prec == 0 else rel_linf_shared(got, ref)
    assert err <= tol, err


@pytest.mark.parametrize("field", ["slab", "shear"])
@pytest.mark.parametrize("recon,flux", [(1, 1), (2, 1), (2, 0)])
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_rough_fields_characteristic_variables_match_oracle(field, recon, flux, prec, tol):
    n = (13, 17, 11)
    prim = ROUGH[field](n)
    cfg = rough_cfg(n, recon, flux, prec, char=1)
    ref, t_o, _ = oracle_run(rough_cfg(n, recon, flux, 0, char=1), prim, 3,
                             key=("rough-char", field, recon, flux))
    got, t = gpu_run(cfg, prim, 3)
    assert t == pytest.approx(t_o, rel=1e-13 if prec == 0 else 1e-6)
    err = rel_linf(got, ref) if prec == 0 else rel_linf_shared(got, ref)
    assert err <= tol, err


# -------------------------------------------------------------- mu = 0 ---

@pytest.mark.parametrize("recon,flux,C", [(0, 0, 0.0), (2, 1, 0.0), (2, 1, 1.0), (1, 1, 0.0)])
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_zero_viscosity_matches_oracle(recon, flux, C, prec, tol):
    """mu = 0: tau = 0 (smooth flux, or full flux with C = 0) -- the Euler
    limit, where exp(-dt/tau) = 0 -- or tau = C |p_l - p_r|/(p_l + p_r) dt
    alone, zero wherever p_l = p_r."""
    n = (12, 10, 9)
    prim = inputs.slab(n, seed=41, axis=0)

    def cfg(p):
        return Config(*n, prec=p, recon=recon, flux=flux, tau_num_C=C, mu_ref=0.0, p_ref=1.0,
                      prandtl=0.72)
    ref, t_o, _ = oracle_run(cfg(0), prim, 3, key=("mu0", recon, flux, C))
    got, t = gpu_run(cfg(prec), prim, 3)
    assert np.isfinite(got).all()
    assert t == pytest.approx(t_o, rel=1e-13 if prec == 0 else 1e-6)
    err = rel_linf(got, ref) if prec == 0 else rel_linf_shared(got, ref)
    assert err <= tol, err


# ------------------------------------------------------- isotropic start ---

def iso_cfg(n, prec, mach_t):
    c = inputs.isotropic_constants(k0=4.0, mach_t=mach_t)
    return Config(n, n, n, prec=prec, recon=2, flux=1, tau_num_C=1.0, prandtl=0.7, visc=1,
                  mu_ref=c["mu0"], T_ref=c["T0"], visc_exp=0.76, p_ref=c["p0"], rho_ref=1.0)


@pytest.mark.parametrize("mach_t", [0.5, 1.0])
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_isotropic_start_matches_oracle(mach_t, prec, tol):
    """The Sec. 3.4 start (seeded solenoidal field, E(k) ~ k^4 exp(-2k^2/k0^2),
    kappa0 = 4) at 32^3: WENO-Z, full flux, tau_num C = 1, mu ~ T^0.76, 2 steps."""
    n = 32
    prim = inputs.isotropic(n, 0, k0=4.0, mach_t=mach_t)
    ref, t_o, _ = oracle_run(iso_cfg(n, 0, mach_t), prim, 2, key=("iso", mach_t))
    got, t = gpu_run(iso_cfg(n, prec, mach_t), prim, 2)
    assert t == pytest.approx(t_o, rel=1e-13 if prec == 0 else 1e-6)
    err = rel_linf(got, ref) if prec == 0 else rel_linf_shared(got, ref)
    print(f"isotropic 32^3 Ma_t {mach_t} prec {prec}: error against the oracle {err:.3e}")
    assert err <= tol, err


# --------------------------------------------------------------- ensemble ---

def test_ensemble_members_match_oracle():
    """A mixed-size, mixed-mode FP64 batch (one graph launch per step): every
    member against the oracle after 3 steps, each with its own CFL step."""
    members = [
        (Config(12, 12, 12, prec=0, recon=0, flux=0, mu_ref=2e-3, p_ref=1.0),
         inputs.random_smooth((12, 12, 12), seed=51, amp=0.2)),
        (Config(13, 10, 9, prec=0, recon=2, flux=1, tau_num_C=1.0, mu_ref=2e-3, p_ref=1.0,
                visc=1, T_ref=1.0, visc_exp=0.76),
         inputs.slab((13, 10, 9), seed=52, axis=0)),
        (iso_cfg(16, 0, 0.5), inputs.isotropic(16, 5, k0=4.0, mach_t=0.5)),
        (Config(9, 11, 8, prec=0, recon=1, flux=0, mu_ref=1e-3, p_ref=1.0, recon_vars=1),
         inputs.shear_layer((9, 11, 8), seed=53)),
    ]
    sims = []
    for cfg, prim in members:
        s = Simulation(cfg)
        s.init_primitive(prim)
        sims.append(s)
    ens = Ensemble(sims)
    ens.step(3)
    for (cfg, prim), s in zip(members, sims):
        ref, t_o, _ = oracle_run(cfg, prim, 3)
        got = s.state()
        assert s.diagnostics()["t"] == pytest.approx(t_o, rel=1e-13)
        assert rel_linf(got, ref) <= FP64_TOL, (cfg, rel_linf(got, ref))
    ens.close()
    for s in sims:
        s.close()
