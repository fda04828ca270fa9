"""Pins of the turbulence-statistics oracle (Sec. 3.1, Sec. 3.4) against closed
forms: trigonometric fields whose cell-centre averages and sixth-order
central differences are known exactly, and the summation-by-parts identity
2 <S^d:S^d> = <|omega|^2> + 4/3 <theta^2> of periodic grids."""
import math

import numpy as np
import pytest

from oracle import conservative
from oracle.turbulence import statistics
from paper_2005_08736_gb300 import inputs

GAMMA = 1.4


def symbol(k: int, h: float) -> float:
    """Fourier symbol of the sixth-order central difference: D e^{ikx} =
    i k g(k, h) e^{ikx} (from the stencil by Euler's formula); g -> 1 as
    h -> 0 with g = 1 - (kh)^6/140 + O(h^8)."""
    return (45 * math.sin(k * h) - 9 * math.sin(2 * k * h) + math.sin(3 * k * h)) / (30 * k * h)


def x_field(n: int, u, p, rho=None, ny: int = 6, nz: int = 6):
    """Primitive state depending on x only, on [0, 2 pi]^3 (n x ny x nz cells)."""
    x = inputs.centres(n, 2 * math.pi)
    prim = np.zeros((5, nz, ny, n))
    prim[0] = 1.0 if rho is None else rho(x)[None, None, :]
    prim[1] = u(x)[None, None, :]
    prim[4] = p(x)[None, None, :]
    return conservative(prim, GAMMA)


@pytest.mark.parametrize("n", [16, 32])
def test_taylor_green_closed_forms(n):
    mu = 1.0 / 1600.0
    cons = conservative(inputs.taylor_green(n), GAMMA)
    s = statistics(cons, gamma=GAMMA, rho0=1.0, mu_ref=mu)
    g = symbol(1, 2 * math.pi / n)
    # <u^2 + v^2>/2 with <sin^2 cos^2 cos^2> = 1/8 per component
    assert s["Ek"] == pytest.approx(0.125, rel=1e-13)
    assert s["u_rms"] == pytest.approx(math.sqrt(0.25 / 3.0), rel=1e-13)
    # omega = g (-cos x sin y sin z, -sin x cos y sin z, 2 sin x sin y cos z): <|omega|^2> = 3/4 g^2
    assert s["zeta"] == pytest.approx(0.375 * g * g, rel=1e-12)
    assert s["omega_rms"] == pytest.approx(math.sqrt(0.75) * g, rel=1e-12)
    # divergence-free: theta = 0 identically, so eps2 = eps3 = eps_d = 0
    assert s["theta_rms"] < 1e-12
    assert abs(s["eps2"]) < 1e-20 and abs(s["eps3"]) < 1e-9 and abs(s["eps_d"]) < 1e-20
    # eps1 = 2 mu/rho0 <S^d:S^d> = mu <|omega|^2> = 2 (mu/rho0) zeta for theta = 0
    assert s["eps1"] == pytest.approx(2 * mu * s["zeta"], rel=1e-12)
    assert s["eps_s"] == pytest.approx(0.75 * mu * g * g, rel=1e-12)
    # d_x u = g cos x cos y cos z: odd moments vanish, <c^4>/<c^2>^2 = (3/8)^3 / (1/8)^2
    assert abs(s["Su"]) < 1e-12
    assert s["Fu"] == pytest.approx(27.0 / 8.0, rel=1e-12)
    assert s["du2_z"] == 0.0
    assert s["rho_rms"] < 1e-14 and s["rho_mean"] == pytest.approx(1.0, rel=1e-15)


def test_enstrophy_sixth_order_convergence():
    # zeta_h / (3/8) = g^2 = 1 - 2 h^6/140 + O(h^8): the error falls 64x per halving.
    errs = []
    for n in (8, 16, 32):
        s = statistics(conservative(inputs.taylor_green(n), GAMMA), gamma=GAMMA)
        errs.append(abs(s["zeta"] / 0.375 - 1.0))
    h = 2 * math.pi / 32
    assert errs[2] == pytest.approx(2 * h ** 6 / 140, rel=0.05)
    assert 50 < errs[1] / errs[2] < 70


def test_compression_wave():
    # u = a sin x, p = p0 + c cos x, rho = 1 + b sin x:
    # theta = a g cos x, omega = 0, S^d:S^d = 2/3 theta^2.
    n, a, b, c, p0, mu = 32, 0.3, 0.05, 0.2, 2.0, 0.01
    cons = x_field(n, lambda x: a * np.sin(x), lambda x: p0 + c * np.cos(x),
                   rho=lambda x: 1.0 + b * np.sin(x))
    s = statistics(cons, gamma=GAMMA, rho0=1.0, mu_ref=mu)
    # the velocity is m / rho = a sin x exactly only up to rounding
    g = symbol(1, 2 * math.pi / n)
    th2 = a * a * g * g / 2
    assert s["theta_rms"] == pytest.approx(math.sqrt(th2), rel=1e-12)
    assert s["eps_d"] == pytest.approx(4.0 / 3.0 * mu * th2, rel=1e-12)
    assert s["eps1"] == pytest.approx(4.0 / 3.0 * mu * th2, rel=1e-12)
    # N = 2 for gamma = 1.4: mu_b = 4/15 mu
    assert s["eps2"] == pytest.approx(4.0 / 15.0 * mu * th2, rel=1e-12)
    assert s["p_theta"] == pytest.approx(c * a * g / 2, rel=1e-12)
    assert s["eps3"] == pytest.approx(-c * a * g / 2, rel=1e-12)
    assert s["eps_s"] < 1e-30 and s["zeta"] < 1e-30
    assert s["rho_rms"] == pytest.approx(b / math.sqrt(2), rel=1e-12)
    assert s["Fu"] == pytest.approx(1.5, rel=1e-12)
    assert abs(s["Su"]) < 1e-12
    # K = 1/2 <rho u^2> = 1/2 <(1 + b sin x) a^2 sin^2 x> = a^2/4
    assert s["K"] == pytest.approx(a * a / 4, rel=1e-12)


def test_skewness_and_flatness_of_two_modes():
    # u = sin x + e sin 2x: d_x u = A cos x + B cos 2x with A = g1, B = 2 e g2;
    # <()^2> = (A^2+B^2)/2, <()^3> = 3 A^2 B / 4,
    # <()^4> = 3 (A^4 + B^4)/8 + 3 A^2 B^2 / 2.
    n, e = 32, 0.4
    h = 2 * math.pi / n
    cons = x_field(n, lambda x: np.sin(x) + e * np.sin(2 * x), lambda x: 5.0 + 0 * x)
    s = statistics(cons, gamma=GAMMA)
    A, B = symbol(1, h), 2 * e * symbol(2, h)
    m2 = (A * A + B * B) / 2
    m3 = 3 * A * A * B / 4
    m4 = 3 * (A ** 4 + B ** 4) / 8 + 1.5 * A * A * B * B
    assert s["du2_x"] == pytest.approx(m2, rel=1e-12)
    assert s["du3_x"] == pytest.approx(m3, rel=1e-12)
    assert s["du4_x"] == pytest.approx(m4, rel=1e-12)
    assert s["Su"] == pytest.approx(m3 / m2 ** 1.5, rel=1e-12)
    assert s["Fu"] == pytest.approx(m4 / m2 ** 2, rel=1e-12)


def test_potential_flow_closed_forms():
    # U = grad phi, phi = sin x sin y sin z (uniform rho, p): the difference
    # operators of different axes commute, so omega = 0 to rounding, and
    # theta = -3 g phi, <theta^2> = 9 g^2 / 8.
    n, mu = 16, 0.01
    x = inputs.centres(n, 2 * math.pi)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    prim = np.zeros((5, n, n, n))
    prim[0] = 1.0
    prim[1] = np.cos(x3) * np.sin(y3) * np.sin(z3)
    prim[2] = np.sin(x3) * np.cos(y3) * np.sin(z3)
    prim[3] = np.sin(x3) * np.sin(y3) * np.cos(z3)
    prim[4] = 3.0
    s = statistics(conservative(prim, GAMMA), gamma=GAMMA, mu_ref=mu)
    g = symbol(1, 2 * math.pi / n)
    assert s["zeta"] < 1e-28 and s["eps_s"] < 1e-30
    assert s["theta_rms"] == pytest.approx(3 * g / math.sqrt(8), rel=1e-12)
    assert s["eps_d"] == pytest.approx(1.5 * mu * g * g, rel=1e-12)
    assert s["eps1"] == pytest.approx(1.5 * mu * g * g, rel=1e-12)


def test_summation_by_parts_identity():
    # On a periodic grid the central-difference operators are skew-adjoint and
    # commute, so 2 <S^d:S^d> = <|omega|^2> + 4/3 <theta^2> exactly:
    # with constant mu, rho0 eps1 = eps_s + eps_d for any field.
    prim = inputs.random_smooth((16, 12, 10), seed=7, amp=0.3, kmax=3)
    s = statistics(conservative(prim, GAMMA), lengths=(2 * np.pi,) * 3, gamma=GAMMA,
                   rho0=1.3, mu_ref=0.02)
    assert 1.3 * s["eps1"] == pytest.approx(s["eps_s"] + s["eps_d"], rel=1e-12)
    assert s["eps_d"] > 1e-3 * s["eps_s"] > 0


def test_power_law_viscosity_scales_with_temperature():
    # uniform T: mu = mu_ref (T/T_ref)^0.76 is a constant factor on eps1, eps_s, eps_d
    prim = inputs.random_smooth((12, 12, 12), seed=3, amp=0.1, kmax=2)
    prim[4] = 2.0 * prim[0]            # p = rho T with T = 2
    cons = conservative(prim, GAMMA)
    a = statistics(cons, gamma=GAMMA, mu_ref=0.01)
    b = statistics(cons, gamma=GAMMA, visc_law=1, mu_ref=0.01, T_ref=1.0, visc_exp=0.76)
    f = 2.0 ** 0.76
    for k in ("eps1", "eps2", "eps_s", "eps_d"):
        assert b[k] == pytest.approx(f * a[k], rel=1e-12)
    assert b["eps3"] == pytest.approx(a["eps3"], rel=1e-12)


def test_reference_density_divides_the_normalised_quantities():
    # Sec. 3.1 / 3.4: E_k, zeta and eps1..eps3 are normalised by rho0; K,
    # eps_s, eps_d and <p theta> are not.  A compressed Taylor-Green field
    # (so that theta != 0) evaluated with rho0 = 1 and rho0 = 2.
    n = 12
    prim = inputs.taylor_green(n)
    x = inputs.centres(n, 2 * math.pi)
    prim[1] += 0.2 * np.sin(x)[None, None, :]
    cons = conservative(prim, GAMMA)
    a = statistics(cons, gamma=GAMMA, rho0=1.0, mu_ref=0.01)
    b = statistics(cons, gamma=GAMMA, rho0=2.0, mu_ref=0.01)
    for k in ("Ek", "zeta", "eps1", "eps2", "eps3"):
        assert abs(a[k]) > 0 and b[k] == pytest.approx(a[k] / 2, rel=1e-14), k
    for k in ("K", "eps_s", "eps_d", "p_theta"):
        assert abs(a[k]) > 0 and b[k] == pytest.approx(a[k], rel=1e-14), k


def test_eps_zeta_of_the_taylor_green_start():
    # zeta = <rho |omega|^2 / 2> / rho0 = (3/8) g^2 for rho = rho0, so
    # eps(zeta) = 2 mu zeta / rho0 = 2 mu (3/8) g^2 / rho0
    n, mu, rho0 = 16, 1.0 / 1600.0, 1.3
    cons = conservative(inputs.taylor_green(n, rho0=rho0), GAMMA)
    s = statistics(cons, gamma=GAMMA, rho0=rho0, mu_ref=mu)
    g = symbol(1, 2 * math.pi / n)
    assert s["zeta"] == pytest.approx(0.375 * g * g, rel=1e-12)
    assert s["eps_zeta"] == pytest.approx(2 * mu * 0.375 * g * g / rho0, rel=1e-12)


def test_dissipation_rate_of_a_quadratic_history_is_exact():
    # second-order differences are exact on a quadratic, on uneven times
    from oracle.turbulence import dissipation_history
    t = np.array([0.0, 0.1, 0.25, 0.3, 0.45, 0.7])
    a, b, c = 0.125, -0.02, 0.003
    stats = [{"Ek": a + b * x + c * x * x, "eps1": 0.01, "eps2": 0.002, "eps3": -0.001} for x in t]
    eps_ek, eps_num = dissipation_history(t, stats)
    assert np.allclose(eps_ek, -(b + 2 * c * t), rtol=0, atol=1e-14)
    assert np.allclose(eps_num, eps_ek - 0.011, rtol=0, atol=1e-14)


def test_decaying_shear_wave_has_no_numerical_dissipation():
    """u = U0 sin(y) e^{-nu t}, v = w = 0, uniform rho and p: an exact solution
    of the incompressible Navier-Stokes equations with E_k = U0^2/4 e^{-2 nu t}.
    Sampled exactly at uneven times, eps(E_k) = 2 nu E_k up to the O(dt^2)
    time differences, eps1 = 2 nu g^2 E_k and eps(zeta) = 2 nu g^2 E_k (g the
    sixth-order difference symbol), eps2 = eps3 = 0; so the numerical
    dissipation eps(E_k) - (eps1 + eps2 + eps3) = 2 nu E_k (1 - g^2) + O(dt^2)
    is tiny against eps(E_k)."""
    from oracle.turbulence import dissipation_history
    n, U0, nu = 32, 0.7, 0.01
    y = inputs.centres(n, 2 * math.pi)
    times = np.array([0.0, 0.05, 0.09, 0.15, 0.2])
    stats = []
    for t in times:
        prim = np.zeros((5, n, n, n))
        prim[0], prim[4] = 1.0, 10.0
        prim[1] = (U0 * math.exp(-nu * t) * np.sin(y))[None, :, None]
        stats.append(statistics(conservative(prim, GAMMA), gamma=GAMMA, rho0=1.0, mu_ref=nu))
    eps_ek, eps_num = dissipation_history(times, stats)
    g2 = symbol(1, 2 * math.pi / n) ** 2
    for t, s, e, en in zip(times, stats, eps_ek, eps_num):
        ek = 0.25 * U0 * U0 * math.exp(-2 * nu * t)
        assert s["Ek"] == pytest.approx(ek, rel=1e-13)
        assert s["eps1"] == pytest.approx(2 * nu * g2 * ek, rel=1e-12)
        assert s["eps_zeta"] == pytest.approx(2 * nu * g2 * ek, rel=1e-12)
        assert abs(s["eps2"]) < 1e-20 and abs(s["eps3"]) < 1e-12
        assert e == pytest.approx(2 * nu * ek, rel=1e-5)
        assert abs(en) < 1e-5 * e
