"""Pins of the oracle's channel statistics (Sec. 3.3), CPU only.

* Laminar Poiseuille flow U = U_c (1 - y^2) with exact cell averages on the
  stretched grid of Sec. 3.3 (uniform rho, T): tau_w = 2 mu U_c at both walls,
  U_b = 2 U_c / 3, the centreline value U_c, and the derived u_tau, Re_tau,
  Re_b, Re_c, C_f in closed form; <u'v'> = 0.
* A density profile rho = 1 + g1 y + g2 y^2: the wall density (mean of the
  two wall rows) and the bulk density (height average) in closed form.
* A shear-free covariance: U = U0 + a cos(kx), V = b cos(kx) gives
  <UV> - <U><V> = a b / 2 in every row.
"""
import math

import numpy as np
import pytest

from oracle.channel import channel_stats
from paper_2005_08736_gb300 import inputs

G = 1.4


def cons_from(rho, U, V, W, p):
    return np.stack([rho, rho * U, rho * V, rho * W, p / (G - 1) + 0.5 * rho * (U * U + V * V + W * W)])


@pytest.mark.parametrize("ny", [24, 31, 64])
def test_poiseuille_statistics_in_closed_form(ny):
    nx, nz, Uc, mu, rho0, p0 = 6, 5, 1.5, 3.0e-4, 1.0, 100 / 1.4
    yf = inputs.channel_faces(ny)
    dy = np.diff(yf)
    # exact cell averages of U_c (1 - y^2)
    ubar = Uc * (1.0 - (yf[:-1] ** 2 + yf[:-1] * yf[1:] + yf[1:] ** 2) / 3.0)
    shape = (nz, ny, nx)
    U = np.broadcast_to(ubar[None, :, None], shape).copy()
    z = np.zeros(shape)
    cons = cons_from(np.full(shape, rho0), U, z, z, np.full(shape, p0))
    out, prof = channel_stats(cons, dy, -1.0, G, mu)
    assert out["tau_w_lower"] == pytest.approx(2 * mu * Uc, rel=1e-11)
    assert out["tau_w_upper"] == pytest.approx(2 * mu * Uc, rel=1e-11)
    assert out["U_b"] == pytest.approx(2 * Uc / 3, rel=1e-13)
    assert out["U_c"] == pytest.approx(Uc, rel=1e-11)
    ut = math.sqrt(2 * mu * Uc / rho0)
    assert out["u_tau"] == pytest.approx(ut, rel=1e-11)
    assert out["Re_tau"] == pytest.approx(rho0 * ut / mu, rel=1e-11)
    nu = mu / rho0
    assert out["Re_b"] == pytest.approx((2 * Uc / 3) * 2 / nu, rel=1e-12)
    assert out["Re_c"] == pytest.approx(Uc / nu, rel=1e-11)
    assert out["C_f"] == pytest.approx(2 * mu * Uc / (0.5 * rho0 * (2 * Uc / 3) ** 2), rel=1e-11)
    assert np.abs(prof["UV"] - prof["U"] * prof["V"]).max() == 0.0


def test_velocity_covariance_in_closed_form():
    nx, ny, nz = 16, 8, 4
    x = 2 * math.pi * (np.arange(nx) + 0.5) / nx
    a, b, U0 = 0.3, 0.2, 1.0
    shape = (nz, ny, nx)
    cx = np.broadcast_to(np.cos(x)[None, None, :], shape)
    U, V = U0 + a * cx, b * cx
    cons = cons_from(np.ones(shape), U, V, np.zeros(shape), np.full(shape, 70.0))
    _, prof = channel_stats(cons, np.full(ny, 2.0 / ny), -1.0, G, 1e-3)
    cov = prof["UV"] - prof["U"] * prof["V"]
    assert np.allclose(cov, a * b / 2, rtol=1e-13, atol=0)


def test_wall_and_bulk_densities_with_a_density_profile():
    # rho = 1 + g1 y + g2 y^2 with exact cell averages on the stretched grid:
    # rho_w, the mean of the two wall rows, keeps only the even part there;
    # rho_b, the height average, is 1 + g2/3.  u_tau, Re_tau and C_f follow
    # with those densities (Poiseuille U).
    ny, nx, nz, Uc, mu, g1, g2 = 32, 4, 3, 1.5, 3.0e-4, 0.2, 0.3
    yf = inputs.channel_faces(ny)
    dy = np.diff(yf)
    a, b = yf[:-1], yf[1:]
    rho_row = 1.0 + g1 * 0.5 * (a + b) + g2 * (a * a + a * b + b * b) / 3.0
    ubar = Uc * (1.0 - (a * a + a * b + b * b) / 3.0)
    shape = (nz, ny, nx)
    rho = np.broadcast_to(rho_row[None, :, None], shape).copy()
    U = np.broadcast_to(ubar[None, :, None], shape).copy()
    z = np.zeros(shape)
    out, prof = channel_stats(cons_from(rho, U, z, z, np.full(shape, 70.0)), dy, -1.0, G, mu)
    rho_w = 1.0 + g2 * (a[0] ** 2 + a[0] * b[0] + b[0] ** 2) / 3.0
    rho_b = 1.0 + g2 / 3.0
    assert out["rho_w"] == pytest.approx(rho_w, rel=1e-13)
    assert out["rho_b"] == pytest.approx(rho_b, rel=1e-13)
    ut = math.sqrt(2 * mu * Uc / rho_w)
    assert out["u_tau"] == pytest.approx(ut, rel=1e-11)
    assert out["Re_tau"] == pytest.approx(rho_w * ut / mu, rel=1e-11)
    assert out["Re_b"] == pytest.approx((2 * Uc / 3) * 2 * rho_b / mu, rel=1e-11)
    assert out["C_f"] == pytest.approx(2 * mu * Uc / (0.5 * rho_b * (2 * Uc / 3) ** 2), rel=1e-11)
