"""Pins of the oracle's interface flux at one Gauss point (CPU only).

* Eq. (5) integrated by brute force over velocity space and time, with the
  slopes re-solved from quadrature moment matrices, against the oracle's
  moment-recursion flux (full flux, Pr = 1).
* A uniform state gives the Euler flux and no time derivative.
* Equal left, right and equilibrium states reduce the full flux to the
  simplified smooth flux (Sec. 2.1, Remark 1).
* Navier-Stokes limits of the smooth flux: shear stress mu du/dy, heat flux
  kappa dT/dx with kappa = mu c_p / Pr (at rest and in a moving gas), and normal stress
  (4/3 mu + mu_b) du/dx with mu_b = 2N/(3(N+3)) mu (Sec. 3.1).
"""
import math

import numpy as np
import pytest

import oracle
from tests.quadrature import GAMMA, K, Maxwell, lin, prim


def cons(rho, u, v, w, p, gamma=GAMMA):
    return np.array([rho, rho * u, rho * v, rho * w,
                     p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)])


def cfg(flux, prandtl=1.0, mu=0.05, C=0.0):
    return oracle.Config(8, 8, 8, flux=flux, prandtl=prandtl, mu_ref=mu, tau_num_C=C)


def euler_flux(Q, gamma=GAMMA):
    rho, U, V, W, lam = prim(Q, gamma)
    p = rho / (2 * lam)
    return np.array([rho * U, rho * U * U + p, rho * U * V, rho * U * W, U * (Q[4] + p)])


def quad_slopes(Q, dQ):
    """Slopes a[3][5] and A[5] from quadrature moment matrices (independent of the oracle)."""
    q = Maxwell(Q)
    psi, vel = q.psi(), q.vel()
    M = np.array([[q.integrate(psi[i] * psi[j]) for j in range(5)] for i in range(5)])
    a = np.array([np.linalg.solve(M, dQ[d]) for d in range(3)])
    rhs = -q.integrate(sum(lin(a[d], psi) * vel[d] for d in range(3))[None, :] * psi)
    A = np.linalg.solve(M, rhs)
    return a, A


def brute_force_full_flux(st, dt, mu, C):
    st = np.asarray(st)
    parts = []
    for s, half in ((0, +1), (1, -1), (2, 0)):
        Q, dQ = st[s, 0], st[s, 1:]
        a, A = quad_slopes(Q, dQ)
        q = Maxwell(Q, half=half)
        psi, vel = q.psi(), q.vel()
        u = vel[0]
        au = sum(lin(a[d], psi) * vel[d] for d in range(3))
        parts.append((q.integrate(u * psi), q.integrate(u * au * psi), q.integrate(u * lin(A, psi) * psi)))
    (Il, Ila, IlA), (Ir, Ira, IrA), (I0, I0a, I0A) = parts
    rho0, _, _, _, lam0 = prim(st[2, 0])
    _, _, _, _, laml = prim(st[0, 0])
    _, _, _, _, lamr = prim(st[1, 0])
    p0, pl, pr = rho0 / (2 * lam0), st[0, 0, 0] / (2 * laml), st[1, 0, 0] / (2 * lamr)
    tau = mu / p0 + C * abs((pl - pr) / (pl + pr)) * dt

    def W(T):
        x, w = np.polynomial.legendre.leggauss(40)
        t = 0.5 * T * (x + 1)
        w = 0.5 * T * w
        e = np.exp(-t / tau)
        tot = np.zeros(5)
        for tk, wk, ek in zip(t, w, e):
            f = ((1 - ek) * I0 + ((tk + tau) * ek - tau) * I0a + (tk - tau + tau * ek) * I0A
                 + ek * (Il - (tau + tk) * Ila - tau * IlA)
                 + ek * (Ir - (tau + tk) * Ira - tau * IrA))
            tot += wk * f
        return tot

    W1, Wh = W(dt), W(0.5 * dt)
    return (4 * Wh - W1) / dt, 4 * (W1 - 2 * Wh) / dt ** 2


def random_point(seed, spread=0.15):
    rng = np.random.default_rng(seed)
    st = np.zeros((3, 4, 5))
    base = dict(rho=1.0, u=0.2, v=-0.1, w=0.15, p=1.0)
    for s in range(3):
        jit = {k: v + spread * rng.uniform(-1, 1) * (1 if k in "rhop" else 1) for k, v in base.items()}
        st[s, 0] = cons(jit["rho"], jit["u"], jit["v"], jit["w"], jit["p"])
        st[s, 1:] = rng.normal(size=(3, 5)) * 0.2
    return st


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_full_flux_matches_brute_force_phase_space_quadrature(seed):
    st = random_point(seed)
    mu, C, dt = 0.04, 1.0, 0.05
    F, dF = oracle.flux_point(cfg(1, 1.0, mu, C), st, dt)
    Fr, dFr = brute_force_full_flux(st, dt, mu, C)
    assert np.allclose(F, Fr, rtol=1e-9, atol=1e-10), (F, Fr)
    assert np.allclose(dF, dFr, rtol=1e-8, atol=1e-9), (dF, dFr)


@pytest.mark.parametrize("flux", [0, 1])
def test_uniform_state_gives_euler_flux(flux):
    st = np.zeros((3, 4, 5))
    Q = cons(1.2, 0.4, -0.3, 0.2, 2.5)
    st[:, 0] = Q
    F, dF = oracle.flux_point(cfg(flux, 0.72, 0.01, 1.0), st, 0.01)
    assert np.allclose(F, euler_flux(Q), rtol=1e-13, atol=1e-13)
    assert np.allclose(dF, 0.0, atol=1e-9)


@pytest.mark.parametrize("seed,prandtl", [(3, 1.0), (4, 0.72)])
def test_full_flux_with_equal_states_is_the_smooth_flux(seed, prandtl):
    st = random_point(seed)
    st[0] = st[2]
    st[1] = st[2]
    for dt in (1e-3, 0.05, 0.5):
        Fs, dFs = oracle.flux_point(cfg(0, prandtl, 0.03), st, dt)
        Ff, dFf = oracle.flux_point(cfg(1, prandtl, 0.03), st, dt)
        assert np.allclose(Ff, Fs, rtol=1e-10, atol=1e-11)
        assert np.allclose(dFf, dFs, rtol=1e-7, atol=1e-8)


MU = 2e-3


def point_with_x_gradient(Q, dQdx):
    st = np.zeros((3, 4, 5))
    st[:, 0] = Q
    st[:, 1] = dQdx
    return st


def test_smooth_flux_shear_stress():
    rho, V, p, s = 1.0, 0.3, 71.43, 0.8          # V(x) with dV/dx = s
    Q = cons(rho, 0.0, V, 0.0, p)
    dQ = np.array([0.0, 0.0, rho * s, 0.0, rho * V * s])   # p uniform
    F, _ = oracle.flux_point(cfg(0, 0.72, MU), point_with_x_gradient(Q, dQ), 1e-3)
    assert F[0] == pytest.approx(0.0, abs=1e-12)
    assert F[1] == pytest.approx(p, rel=1e-13)
    assert F[2] == pytest.approx(-MU * s, rel=1e-9)
    assert F[4] == pytest.approx(-MU * s * V, rel=1e-9)


@pytest.mark.parametrize("prandtl", [1.0, 0.72])
def test_heat_flux_in_a_moving_gas(prandtl):
    # Galilean invariance: a temperature gradient at uniform pressure carried
    # by a uniform velocity (U, V, W) has no viscous stress, so the energy
    # flux is the Euler one plus -mu c_p / Pr dT/dx, with the Prandtl
    # correction measured in the frame of the gas.
    p, T, s = 2.0, 1.6, 0.5                      # T(x) with dT/dx = s, p uniform
    U, V, W = 0.7, -0.4, 0.3
    rho = p / T
    Q = cons(rho, U, V, W, p)
    drho = -rho * s / T
    dQ = np.array([drho, U * drho, V * drho, W * drho, 0.5 * (U * U + V * V + W * W) * drho])
    F, _ = oracle.flux_point(cfg(0, prandtl, MU), point_with_x_gradient(Q, dQ), 1e-3)
    cp = (K + 5) / 2.0
    E = euler_flux(Q)
    assert F[:4] == pytest.approx(E[:4], rel=1e-12, abs=1e-12)
    assert F[4] == pytest.approx(E[4] - MU * cp / prandtl * s, rel=1e-10)


@pytest.mark.parametrize("flux", [0, 1])
def test_shear_stress_follows_the_power_law_viscosity(flux):
    # Sec. 3.4: mu = mu_ref (T / T_ref)^0.76; the stress of a uniform shear at
    # a temperature T = 2.5 T_ref carries that viscosity (both fluxes).
    rho, V, T_ref, s = 1.0, 0.3, 0.8, 0.8
    p = 2.5 * T_ref * rho
    Q = cons(rho, 0.0, V, 0.0, p)
    dQ = np.array([0.0, 0.0, rho * s, 0.0, rho * V * s])
    c = oracle.Config(8, 8, 8, flux=flux, prandtl=0.7, mu_ref=MU, visc_law=1, T_ref=T_ref,
                      visc_exp=0.76)
    F, _ = oracle.flux_point(c, point_with_x_gradient(Q, dQ), 1e-4)
    mu = MU * 2.5 ** 0.76
    assert F[2] == pytest.approx(-mu * s, rel=1e-8)
    assert F[4] == pytest.approx(-mu * s * V, rel=1e-8)


@pytest.mark.parametrize("prandtl", [1.0, 0.72, 0.7])
def test_smooth_flux_heat_flux(prandtl):
    p, T, s = 2.0, 1.6, 0.5                      # T(x) with dT/dx = s, p uniform
    rho = p / T
    Q = cons(rho, 0.0, 0.0, 0.0, p)
    dQ = np.array([-rho * s / T, 0.0, 0.0, 0.0, 0.0])
    F, _ = oracle.flux_point(cfg(0, prandtl, MU), point_with_x_gradient(Q, dQ), 1e-3)
    cp = (K + 5) / 2.0
    assert F[4] == pytest.approx(-MU * cp / prandtl * s, rel=1e-9)
    assert F[1] == pytest.approx(p, rel=1e-13)


def test_smooth_flux_normal_stress_and_bulk_viscosity():
    rho, p, s = 1.0, 5.0, 0.7                    # U(x) with dU/dx = s at U = 0
    Q = cons(rho, 0.0, 0.0, 0.0, p)
    dQ = np.array([0.0, rho * s, 0.0, 0.0, 0.0])
    F, _ = oracle.flux_point(cfg(0, 0.72, MU), point_with_x_gradient(Q, dQ), 1e-3)
    mu_b = 2 * K / (3 * (K + 3)) * MU
    assert F[1] == pytest.approx(p - (4.0 / 3.0 * MU + mu_b) * s, rel=1e-12)


@pytest.mark.parametrize("flux", [0, 1])
def test_normal_stress_work_in_a_moving_gas(flux):
    # u = U + s x with V, W uniform, rho and p uniform: the stress is the
    # normal one, (4/3 mu + mu_b) s, it does work U (4/3 mu + mu_b) s on the
    # energy flux, and no heat flows (T uniform), so the Prandtl correction,
    # taken in the frame of the gas, adds nothing (Pr = 0.72 here).
    rho, p, s = 1.0, 5.0, 0.7
    U, V, W = 0.6, -0.5, 0.25
    Q = cons(rho, U, V, W, p)
    dQ = np.array([0.0, rho * s, 0.0, 0.0, rho * U * s])
    F, _ = oracle.flux_point(cfg(flux, 0.72, MU), point_with_x_gradient(Q, dQ), 1e-4)
    sxx = (4.0 / 3.0 * MU + 2 * K / (3 * (K + 3)) * MU) * s
    E = euler_flux(Q)
    assert F[0] == pytest.approx(E[0], rel=1e-12)
    assert F[1] == pytest.approx(E[1] - sxx, rel=1e-10)
    assert F[2] == pytest.approx(E[2], rel=1e-10)
    assert F[3] == pytest.approx(E[3], rel=1e-10)
    assert F[4] == pytest.approx(E[4] - U * sxx, rel=1e-10)
