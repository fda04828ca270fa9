"""Pins of the oracle's streamwise force (Sec. 3.3).

* Constant f_x on a uniform state: the fluxes vanish, so the step must give
  the exact solution of d(rho U)/dt = rho f, d(rho E)/dt = rho U f (rho U is
  linear in t, so the trapezoidal force update is exact).
* Constant mass flux: after every step the volume integral of rho U equals
  the target; the force applied equals the one computed from the unforced
  step, and the constant-force step with that f_x gives the same state.
"""
import numpy as np
import pytest

import oracle
from paper_2005_08736_gb300 import inputs

CH = dict(ly=2.0, y0=-1.0, y_stretch=1, stretch_b=2.0, bc_y=1, T_wall=100 / 1.4,
          mu_ref=0.0541 / 180, cfl=0.5)


def test_constant_force_on_uniform_state_is_exact():
    n, f, dt = 6, 0.05, 0.01
    rho, U, p = 1.3, 0.4, 2.0
    s = oracle.Solver(oracle.Config(n, n, n, force_x=f, mu_ref=0.01))
    prim = np.zeros((5, n, n, n))
    prim[0], prim[1], prim[4] = rho, U, p
    Q0 = oracle.conservative(prim, 1.4)
    s.set_state(Q0)
    s.step(1, dt)
    Q = s.state()
    assert np.allclose(Q[0], rho, rtol=1e-14)
    assert np.allclose(Q[1], rho * U + rho * f * dt, rtol=1e-14)
    E_exact = Q0[4] + rho * U * f * dt + 0.5 * rho * f * f * dt * dt
    assert np.allclose(Q[4], E_exact, rtol=1e-14)
    assert s.last_force == f


def channel_solver(n, **kw):
    nx, ny, nz = n
    c = oracle.Config(nx, ny, nz, lx=2 * np.pi, lz=np.pi, **CH, **kw)
    s = oracle.Solver(c)
    s.set_state(oracle.conservative(inputs.channel(nx, ny, nz, 0), 1.4))
    return s


def volume_integral(s, v):
    wx, wy, wz = (s.widths(d) for d in range(3))
    vol = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    return float((s.state()[v] * vol).sum()), float(vol.sum())


def test_mass_flux_force_holds_the_target():
    n = (6, 12, 6)
    target = 1.02
    s = channel_solver(n, force_mode=1, mass_flux=target)
    for _ in range(3):
        s.step(1)
        m, vol = volume_integral(s, 1)
        assert m / vol == pytest.approx(target, rel=1e-13)


def test_mass_flux_force_equals_the_closed_form_and_the_constant_force_step():
    n = (6, 12, 6)
    target, dt = 1.05, 2e-3
    forced = channel_solver(n, force_mode=1, mass_flux=target)
    forced.step(1, dt)
    f = forced.last_force
    # the unforced step gives (rho U)~ and rho~; f follows from Sec. 3.3
    free = channel_solver(n)
    rho_n, _ = volume_integral(free, 0)
    free.step(1, dt)
    m_t, vol = volume_integral(free, 1)
    rho_t, _ = volume_integral(free, 0)
    f_ref = (target * vol - m_t) / (dt * 0.5 * (rho_n + rho_t))
    assert f == pytest.approx(f_ref, rel=1e-12)
    assert f > 0
    # the constant-force step with the same f_x gives the same state
    const = channel_solver(n, force_x=f)
    const.step(1, dt)
    assert np.allclose(const.state(), forced.state(), rtol=1e-14, atol=0)
