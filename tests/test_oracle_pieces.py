"""Pins of the oracle's single pieces against quadrature, closed forms and
textbook special cases (CPU only).

Each test recomputes what one oracle function returns by a route that shares
nothing with it: brute-force velocity quadrature instead of moment
recursions, numerical time integration instead of the closed-form time
integrals, polynomial data with known exact answers, and the Navier-Stokes
limits of the BGK flux (Cao, Pan & Xu, Sec. 2.1 and Sec. 3.1).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from tests.quadrature import GAMMA, K, Maxwell, lin, prim


def cons(rho, u, v, w, p, gamma=GAMMA):
    return np.array([rho, rho * u, rho * v, rho * w,
                     p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)])


# ---------------------------------------------------------------- moments ---

@pytest.mark.parametrize("U,lam", [(0.3, 0.7), (-1.2, 2.0), (0.0, 0.05), (2.5, 0.4), (-0.05, 30.0)])
def test_moments_match_quadrature(U, lam):
    m = oracle.moments(U, 0.4, -0.7, lam, 2.0)
    s = 1 / math.sqrt(lam)
    phi = lambda x: math.sqrt(lam / math.pi) * math.exp(-lam * (x - U) ** 2)
    for n in range(8):
        pos = integrate.quad(lambda x: x ** n * phi(x), 0.0, U + 40 * s if U > 0 else 40 * s,
                             epsabs=0, epsrel=1e-13, limit=200)[0]
        neg = integrate.quad(lambda x: x ** n * phi(x), U - 40 * s if U < 0 else -40 * s, 0.0,
                             epsabs=0, epsrel=1e-13, limit=200)[0]
        scale = max(1.0, abs(U) + s) ** n
        assert m["up"][n] == pytest.approx(pos, abs=1e-12 * scale)
        assert m["un"][n] == pytest.approx(neg, abs=1e-12 * scale)
        assert m["uf"][n] == pytest.approx(pos + neg, abs=1e-12 * scale)
    # v and w: full-line Gaussian moments of mean 0.4 and -0.7.
    for mean, key in ((0.4, "v"), (-0.7, "w")):
        for n in range(8):
            ref = integrate.quad(lambda x: x ** n * math.sqrt(lam / math.pi) * math.exp(-lam * (x - mean) ** 2),
                                 mean - 40 * s, mean + 40 * s, epsabs=0, epsrel=1e-13, limit=200)[0]
            assert m[key][n] == pytest.approx(ref, abs=1e-12 * max(1.0, abs(mean) + s) ** n)


@pytest.mark.parametrize("Kdof", [2, 3])
def test_internal_moments_match_radial_quadrature(Kdof):
    lam = 0.37
    m = oracle.moments(0.0, 0.0, 0.0, lam, float(Kdof))
    # int (xi^2)^k (lam/pi)^{K/2} exp(-lam xi^2) d^K xi, in polar form.
    area = 2 * math.pi if Kdof == 2 else 4 * math.pi
    for k in range(4):
        ref = area * (lam / math.pi) ** (Kdof / 2) * integrate.quad(
            lambda r: r ** (2 * k + Kdof - 1) * math.exp(-lam * r * r), 0, 60, epsabs=0, epsrel=1e-13)[0]
        assert m["xi"][k] == pytest.approx(ref, rel=1e-12)


# ------------------------------------------------------- slopes and A ---

STATES = [cons(1.0, 0.2, -0.1, 0.05, 0.8), cons(0.7, -0.6, 0.3, 0.2, 1.3), cons(1.3, 0.0, 0.0, 0.0, 71.4)]


@pytest.mark.parametrize("Q", STATES)
def test_slope_solve_matches_quadrature_moment_matrix(Q):
    rng = np.random.default_rng(3)
    b = rng.normal(size=5)
    a = oracle.slope(Q, GAMMA, b)
    q = Maxwell(Q)
    psi = q.psi()
    M = np.array([[q.integrate(psi[i] * psi[j]) for j in range(5)] for i in range(5)]) / q.rho
    assert np.allclose(M @ a, b, rtol=1e-11, atol=1e-11 * np.abs(b).max())
    assert np.allclose(a, np.linalg.solve(M, b), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("Q", STATES)
def test_slope_solve_matches_closed_form(Q):
    # Closed-form inverse of the 5x5 moment matrix, derived by hand from
    # <psi_i psi_j> with U, V, W, lambda and K internal degrees of freedom.
    rng = np.random.default_rng(4)
    b = rng.normal(size=5)
    rho, U, V, W, lam = prim(Q)
    q2 = U * U + V * V + W * W
    a5 = 4 * lam * lam / (K + 3) * (2 * b[4] - 2 * U * b[1] - 2 * V * b[2] - 2 * W * b[3]
                                     + (q2 - (K + 3) / (2 * lam)) * b[0])
    a4 = 2 * lam * (b[3] - W * b[0]) - W * a5
    a3 = 2 * lam * (b[2] - V * b[0]) - V * a5
    a2 = 2 * lam * (b[1] - U * b[0]) - U * a5
    a1 = b[0] - U * a2 - V * a3 - W * a4 - 0.5 * a5 * (q2 + (K + 3) / (2 * lam))
    a = oracle.slope(Q, GAMMA, b)
    assert np.allclose(a, [a1, a2, a3, a4, a5], rtol=1e-10, atol=1e-10 * np.abs(a).max())


@pytest.mark.parametrize("Q", STATES[:2])
def test_kinetic_conditions_hold_by_quadrature(Q):
    rng = np.random.default_rng(5)
    dQ = rng.normal(size=(3, 5)) * 0.3
    a, A = oracle.kinetic(Q, dQ, GAMMA)
    q = Maxwell(Q)
    psi, vel = q.psi(), q.vel()
    for d in range(3):
        got = q.integrate(lin(a[d], psi)[None, :] * psi)
        assert np.allclose(got, dQ[d], atol=1e-11)
    # <a_1 u + a_2 v + a_3 w + A> = 0 (moments against psi).
    expr = sum(lin(a[d], psi) * vel[d] for d in range(3)) + lin(A, psi)
    assert np.allclose(q.integrate(expr[None, :] * psi), 0.0, atol=1e-11)


# ------------------------------------------------------ compatibility Q0 ---

def test_compatibility_matches_half_space_quadrature():
    Ql = cons(1.1, 0.3, 0.1, -0.2, 0.9)
    Qr = cons(0.8, -0.4, 0.2, 0.1, 1.2)
    Q0 = oracle.compat(Ql, Qr, GAMMA)
    ql, qr = Maxwell(Ql, half=+1), Maxwell(Qr, half=-1)
    ref = ql.integrate(ql.psi()) + qr.integrate(qr.psi())
    assert np.allclose(Q0, ref, rtol=1e-12, atol=1e-13)


def test_compatibility_of_equal_states_is_the_state():
    Q = cons(0.9, 0.35, -0.2, 0.1, 2.0)
    assert np.allclose(oracle.compat(Q, Q, GAMMA), Q, rtol=1e-14, atol=1e-14)


# ------------------------------------------------------- time integrals ---

@pytest.mark.parametrize("T,tau", [(1e-2, 3e-3), (1e-3, 5e-2), (0.5, 0.5), (2e-3, 1e-6)])
def test_time_integrals_match_numerical_integration(T, tau):
    q = oracle.time_integrals(T, tau)
    e = lambda t: math.exp(-t / tau)
    fns = [lambda t: 1 - e(t),
           lambda t: (t + tau) * e(t) - tau,
           lambda t: t - tau + tau * e(t),
           lambda t: e(t),
           lambda t: -(tau + t) * e(t),
           lambda t: -tau * e(t)]
    for k, f in enumerate(fns):
        ref = integrate.quad(f, 0, T, epsabs=0, epsrel=1e-13, limit=200, points=[min(T, 10 * tau)])[0]
        assert q[k] == pytest.approx(ref, rel=1e-9, abs=1e-15 * max(T, T * T))


def test_time_integrals_euler_limit():
    q = oracle.time_integrals(0.01, 0.0)
    assert np.allclose(q, [0.01, 0.0, 0.5e-4, 0.0, 0.0, 0.0], atol=0)


# ---------------------------------------------------------------- WENO5 ---

def cell_avgs(poly, centres, h=1.0):
    P = np.polyint(poly)
    return np.array([(np.polyval(P, c + h / 2) - np.polyval(P, c - h / 2)) / h for c in centres])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_weno5_exact_on_quadratics(mode):
    rng = np.random.default_rng(7)
    for _ in range(5):
        poly = rng.normal(size=3)
        q = cell_avgs(poly, np.arange(-2, 3))
        assert oracle.weno5_right(q, mode) == pytest.approx(np.polyval(poly, 0.5), abs=1e-12)
        assert oracle.weno5_left(q, mode) == pytest.approx(np.polyval(poly, -0.5), abs=1e-12)


def test_weno5_linear_weights_exact_on_quartics():
    rng = np.random.default_rng(8)
    for _ in range(5):
        poly = rng.normal(size=5)
        q = cell_avgs(poly, np.arange(-2, 3))
        assert oracle.weno5_right(q, 0) == pytest.approx(np.polyval(poly, 0.5), abs=1e-12)
        assert oracle.weno5_left(q, 0) == pytest.approx(np.polyval(poly, -0.5), abs=1e-12)


@pytest.mark.parametrize("mode,order", [(2, 4.6), (1, 4.6)])
def test_weno5_nonlinear_weights_converge_to_linear(mode, order):
    # On smooth data away from critical points the nonlinear weights tend to
    # the linear ones; the reconstruction error is then fifth order.
    errs = []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        x = 0.3 + h * np.arange(-2, 3)
        q = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h  # averages of sin
        errs.append(abs(oracle.weno5_right(q, mode) - math.sin(0.3 + h / 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > order, (errs, rates)


def weno5_right_by_definition(q, mode):
    """The WENO5 value at the right end of the centre cell built from the
    definitions (Jiang & Shu; Borges et al. for WENO-Z), cell units: each
    candidate is the quadratic whose averages over its three cells are the
    data (a 3x3 solve), its indicator is the integral over the centre cell of
    p'^2 + p''^2 (Gauss-Legendre quadrature, exact here), and the weights are
    d_k / (eps + beta_k)^2 (WENO-JS, eps 1e-6) or d_k (1 + |beta_0 - beta_2| /
    (beta_k + eps)) (WENO-Z, eps 1e-20), normalised."""
    xg, wg = np.polynomial.legendre.leggauss(4)
    xg, wg = 0.5 * xg, 0.5 * wg                  # the centre cell [-1/2, 1/2]
    d = np.array([0.1, 0.6, 0.3])
    vals, beta = [], []
    for k in range(3):                           # stencils {i-2..i}, {i-1..i+1}, {i..i+2}
        cells = np.arange(3) + k - 2
        # average of s^m over [c - 1/2, c + 1/2]
        A = np.array([[((c + 0.5) ** (m + 1) - (c - 0.5) ** (m + 1)) / (m + 1) for m in range(3)]
                      for c in cells])
        a = np.linalg.solve(A, q[k:k + 3])
        vals.append(a[0] + a[1] * 0.5 + a[2] * 0.25)
        d1 = a[1] + 2 * a[2] * xg
        beta.append(float(np.sum(wg * (d1 ** 2 + (2 * a[2]) ** 2))))
    beta = np.array(beta)
    if mode == 1:
        alpha = d / (1e-6 + beta) ** 2
    else:
        alpha = d * (1 + abs(beta[0] - beta[2]) / (beta + 1e-20))
    return float(np.dot(alpha / alpha.sum(), vals))


@pytest.mark.parametrize("mode", [1, 2])
def test_weno5_matches_its_definition_on_random_data(mode):
    rng = np.random.default_rng(5)
    for scale in (1.0, 0.05, 3e-3):              # rough to nearly smooth data
        for _ in range(40):
            q = 1.0 + scale * rng.normal(size=5)
            ref = weno5_right_by_definition(q, mode)
            assert oracle.weno5_right(q, mode) == pytest.approx(ref, rel=1e-12, abs=1e-13)
            # the left end value is the mirror image
            refl = weno5_right_by_definition(q[::-1].copy(), mode)
            assert oracle.weno5_left(q, mode) == pytest.approx(refl, rel=1e-12, abs=1e-13)


def test_weno_z_is_linear_where_the_outer_indicators_agree():
    # Data symmetric about the centre cell give beta_0 = beta_2, so the
    # WENO-Z indicator |beta_0 - beta_2| vanishes and its weights are the
    # linear ones; WENO-JS weights still follow beta_k and differ.
    for q in ([0.3, 1.1, -0.4, 1.1, 0.3], [2.0, 0.5, 1.0, 0.5, 2.0]):
        q = np.array(q)
        for side in (oracle.weno5_right, oracle.weno5_left):
            lin = side(q, 0)
            assert side(q, 2) == pytest.approx(lin, rel=1e-14, abs=1e-14)
            assert abs(side(q, 1) - lin) > 1e-3


@pytest.mark.parametrize("mode", [1, 2])
def test_weno5_non_oscillatory_at_a_step(mode):
    q = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    assert abs(oracle.weno5_right(q, mode)) < 1e-5       # smooth left stencil chosen
    q = np.array([0.0, 0.0, 1.0, 1.0, 1.0])
    assert abs(oracle.weno5_right(q, mode) - 1.0) < 1e-5
    assert oracle.weno5_right(q, 0) > 1.0                # linear weights overshoot


def test_weno5_constant_data():
    for mode in (0, 1, 2):
        assert oracle.weno5_right(np.full(5, 3.25), mode) == 3.25


# ------------------------------------------------------- tangential recon ---

GS = np.array([-0.5, 0.5]) / math.sqrt(3.0)


def test_tangential_quartic_exact():
    rng = np.random.default_rng(9)
    for _ in range(5):
        poly = rng.normal(size=5)
        f = cell_avgs(poly, np.arange(-2, 3))
        val, der = oracle.tangential(f, 0)
        assert np.allclose(val, np.polyval(poly, GS), atol=1e-12)
        assert np.allclose(der, np.polyval(np.polyder(poly), GS), atol=1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_tangential_weno_quadratic_exact(mode):
    rng = np.random.default_rng(10)
    for _ in range(5):
        poly = rng.normal(size=3)
        f = cell_avgs(poly, np.arange(-2, 3))
        val, der = oracle.tangential(f, mode)
        assert np.allclose(val, np.polyval(poly, GS), atol=1e-12)
        assert np.allclose(der, np.polyval(np.polyder(poly), GS), atol=1e-12)


# ---------------------------------------------------------------- S2O4 ---

def test_s2o4_on_linear_ode_is_the_fourth_order_taylor_polynomial():
    # y' = lam y: L = lam y and dL/dt = lam^2 y.  Eq. (6) must give
    # y^{n+1} = (1 + z + z^2/2 + z^3/6 + z^4/24) y^n, z = lam dt.
    for lam, dt in [(-1.3, 0.1), (0.7, 0.25), (-4.0, 0.5)]:
        y = 1.7
        ys = oracle.s2o4_stage1(y, lam * y, lam * lam * y, dt)
        y1 = oracle.s2o4_stage2(y, lam * y, lam * lam * y, lam * lam * ys, dt)
        z = lam * dt
        assert y1 == pytest.approx(y * (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24), rel=1e-14)
