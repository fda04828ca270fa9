"""Pins of the oracle's dual-number tangent run (CPU only).

The tangent build compiles the unchanged oracle source with forward-mode dual
numbers as its scalar type, so one run gives Q^n and dQ^n/dQ^0 along a
direction v (dt held fixed).  It is pinned against the plain oracle:

* its value part equals the plain FP64 oracle bit for bit (same double
  operations, no FP contraction), in every mode, with walls, stretching and
  the constant-mass-flux force;
* its tangent equals central differences of the plain oracle where the step
  is differentiable (linear weights, WENO-JS, smooth and full flux, the
  characteristic variables of Remark 1, the channel of Sec. 3.3), with the
  O(h^2) convergence of a correct derivative;
* where the step has kinks (WENO-Z's |beta0 - beta2| and the numerical
  collision time's |p_l - p_r|), central differences approach the tangent as
  h shrinks.

A wrong derivative rule (erfc of the half-space moments, the power-law
viscosity, sqrt, exp of the time integrals, the quotient rule) breaks the
second group.
"""
import numpy as np
import pytest

import oracle
from paper_2005_08736_gb300 import inputs

N = (8, 7, 6)
DT = 0.05


def periodic_case(recon, flux, C=0.0, char=0):
    cfg = oracle.Config(*N, recon=recon, flux=flux, tau_num_C=C, char_recon=char, visc_law=1,
                        mu_ref=5e-3, prandtl=0.7)
    q0 = oracle.conservative(inputs.random_smooth(N, seed=3, amp=0.1, kmax=1), 1.4)
    return cfg, q0, DT


def channel_case():
    n = (6, 8, 6)
    cfg = oracle.Config(*n, lx=2 * np.pi, ly=2.0, y0=-1.0, lz=np.pi, y_stretch=1, stretch_b=2.0,
                        bc_y=1, T_wall=1 / 1.4, mu_ref=0.01, force_mode=1, mass_flux=0.8)
    prim = inputs.channel(*n, 0)
    prim[4] = 1 / 1.4  # c0 = 1: a moderate Mach number keeps dt and the test small
    return cfg, oracle.conservative(prim, 1.4), 0.002


def direction(q0, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(q0.shape) * np.abs(q0).max(axis=(1, 2, 3), keepdims=True)


def plain(cfg, q, dt, steps):
    s = oracle.Solver(cfg)
    s.set_state(q)
    s.step(steps, dt)
    return s.state()


def tangent_run(cfg, q0, v, dt, steps):
    t = oracle.TangentSolver(cfg)
    t.set_state(q0, v)
    t.step(steps, dt)
    return t.state(), t.tangent()


def central(cfg, q0, v, dt, steps, h):
    return (plain(cfg, q0 + h * v, dt, steps) - plain(cfg, q0 - h * v, dt, steps)) / (2 * h)


CASES = {
    "linear-smooth": lambda: periodic_case(0, 0),
    "wenojs-smooth": lambda: periodic_case(1, 0),
    "wenojs-full-char": lambda: periodic_case(1, 1, char=1),
    "wenoz-full-taunum": lambda: periodic_case(2, 1, C=1.0),
    "channel-massflux": channel_case,
}


@pytest.mark.parametrize("name", list(CASES))
def test_tangent_values_equal_the_plain_oracle_bitwise(name):
    cfg, q0, dt = CASES[name]()
    val, _ = tangent_run(cfg, q0, direction(q0), dt, 2)
    assert np.array_equal(val, plain(cfg, q0, dt, 2))


@pytest.mark.parametrize("name", ["linear-smooth", "wenojs-smooth", "wenojs-full-char",
                                  "channel-massflux"])
def test_tangent_equals_central_differences_where_smooth(name):
    cfg, q0, dt = CASES[name]()
    v = direction(q0)
    _, tan = tangent_run(cfg, q0, v, dt, 2)
    scale = np.abs(tan).max()
    e1 = np.abs(central(cfg, q0, v, dt, 2, 1e-5) - tan).max() / scale
    e2 = np.abs(central(cfg, q0, v, dt, 2, 1e-6) - tan).max() / scale
    assert e2 <= 1e-6, (e1, e2)
    # O(h^2): a tenth of the step gives about a hundredth of the error, until
    # round-off takes over
    assert e2 <= max(0.05 * e1, 2e-9), (e1, e2)


def test_tangent_is_the_limit_of_differences_across_kinks():
    cfg, q0, dt = CASES["wenoz-full-taunum"]()
    v = direction(q0)
    _, tan = tangent_run(cfg, q0, v, dt, 2)
    scale = np.abs(tan).max()
    errs = [np.abs(central(cfg, q0, v, dt, 2, h) - tan).max() / scale for h in (1e-5, 1e-8)]
    assert errs[1] < 0.01 * errs[0] and errs[1] <= 2e-6, errs


def test_tangent_run_rejects_a_cfl_time_step():
    cfg, q0, _ = CASES["linear-smooth"]()
    t = oracle.TangentSolver(cfg)
    t.set_state(q0, direction(q0))
    with pytest.raises(ValueError):
        t.step(1, 0.0)
