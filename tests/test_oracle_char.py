"""Pins of the oracle's characteristic-variable reconstruction (Sec. 2.1,
Remark 1): the basis against the Jacobian of the Euler flux (complex-step
derivatives), the invariance of linear-weight reconstruction under the
projection, exact velocity and pressure across a contact discontinuity, and
the separate reconstruction of superposed characteristic fields (normal end
values and tangential Gauss-point values)."""
import numpy as np
import pytest

import oracle
from paper_2005_08736_gb300 import inputs

GAMMA = 1.4


def euler_flux_local(Q, gamma=GAMMA):
    """Euler flux along the first velocity component of a local-frame state."""
    rho, m, n, l, E = Q
    u, v, w = m / rho, n / rho, l / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w))
    return np.array([m, m * u + p, m * v, m * w, u * (E + p)])


def jacobian(Q):
    """dF/dQ by complex-step differentiation (exact to rounding)."""
    h = 1e-30
    J = np.empty((5, 5))
    for k in range(5):
        Qc = np.array(Q, dtype=complex)
        Qc[k] += 1j * h
        J[:, k] = euler_flux_local(Qc).imag / h
    return J


def state(rho, u, v, w, p):
    return oracle.conservative(np.array([rho, u, v, w, p], dtype=float), GAMMA)


@pytest.mark.parametrize("prim", [(1.0, 0.3, -0.2, 0.1, 1.0), (0.7, -1.4, 0.5, 2.0, 0.3),
                                  (1.2, 0.0, 0.0, 0.0, 71.4)])
def test_basis_diagonalises_the_euler_jacobian(prim):
    Q = state(*prim)
    R, L = oracle.char_basis(Q, GAMMA)
    rho, u, v, w, p = prim
    c = np.sqrt(GAMMA * p / rho)
    lam = np.array([u - c, u, u, u, u + c])
    J = jacobian(Q)
    scale = np.abs(J).max() * np.abs(R).max()
    assert np.abs(J @ R - R * lam[None, :]).max() <= 1e-13 * scale
    assert np.abs(L @ R - np.eye(5)).max() <= 1e-13 * np.abs(R).max() * np.abs(L).max()


def random_cells(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    prim = np.stack([1 + 0.3 * rng.uniform(-1, 1, 6), rng.uniform(-1, 1, 6), rng.uniform(-1, 1, 6),
                     rng.uniform(-1, 1, 6), 1 + 0.3 * rng.uniform(-1, 1, 6)])
    return oracle.conservative(prim, GAMMA).T.copy()  # [6][5]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_linear_weights_are_invariant_under_the_projection(seed):
    qc = random_cells(seed)
    a = oracle.normal_end_values(qc, 0, 0)
    b = oracle.normal_end_values(qc, 0, 1)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("mode", [1, 2])
def test_contact_discontinuity_keeps_velocity_and_pressure(mode):
    # rho jumps, (u, v, w, p) uniform: the jump lies along the entropy
    # eigenvector at every state with this velocity, so in characteristic
    # variables only one component varies and u, p stay exactly uniform.
    U, p = (0.4, -0.3, 0.2), 2.0
    rho = [1.0, 1.0, 1.0, 0.2, 0.2, 0.2]
    qc = np.array([state(r, *U, p) for r in rho])
    e = oracle.normal_end_values(qc, mode, 1)
    u = e[:, 1] / e[:, 0]
    pe = 0.4 * (e[:, 4] - 0.5 * (e[:, 1] ** 2 + e[:, 2] ** 2 + e[:, 3] ** 2) / e[:, 0])
    assert np.abs(u - U[0]).max() <= 1e-13
    assert np.abs(pe - p).max() <= 1e-13 * p


@pytest.mark.parametrize("mode", [1, 2])
def test_two_superposed_fields_are_reconstructed_separately(mode):
    # Data Q_s = Qm + a_s r1 + b_s r5 in the basis of Qm, with a_2 + a_3 =
    # b_2 + b_3 = 0 so that Qm is the mean of the two cells beside the face: a
    # jump in the u - c field and a smooth u + c field.  In characteristic
    # variables each end value is Qm + WENO(a) r1 + WENO(b) r5 with the scalar
    # WENO of each profile; the shear and entropy components stay zero.  The
    # component-wise reconstruction mixes the two profiles.
    Qm = state(1.0, 0.3, -0.2, 0.1, 1.0)
    R, L = oracle.char_basis(Qm, GAMMA)
    a = np.array([0.2, 0.2, 0.2, -0.2, -0.2, -0.2])
    b = 0.05 * np.array([-2.5, -1.5, -0.5, 0.5, 1.5, 2.5]) ** 3
    qc = Qm[None, :] + a[:, None] * R[:, 0][None, :] + b[:, None] * R[:, 4][None, :]

    def scalar(f):
        return np.array([oracle.weno5_right(f[0:5], mode), oracle.weno5_left(f[0:5], mode),
                         oracle.weno5_left(f[1:6], mode), oracle.weno5_right(f[1:6], mode)])
    ch = (L @ (oracle.normal_end_values(qc, mode, 1) - Qm[None, :]).T).T
    assert np.abs(ch[:, 1:4]).max() <= 1e-13
    assert np.abs(ch[:, 0] - scalar(a)).max() <= 1e-13
    assert np.abs(ch[:, 4] - scalar(b)).max() <= 1e-13
    cw = (L @ (oracle.normal_end_values(qc, mode, 0) - Qm[None, :]).T).T
    assert np.abs(cw[:, 1:4]).max() > 1e-6 or np.abs(cw[:, 4] - scalar(b)).max() > 1e-6


@pytest.mark.parametrize("mode", [1, 2])
def test_tangential_reconstruction_separates_superposed_fields(mode):
    Qm = state(1.1, -0.4, 0.3, 0.2, 0.8)
    R, L = oracle.char_basis(Qm, GAMMA)
    a = np.array([0.1, 0.1, 0.1, -0.3, -0.3])
    b = 0.02 * np.array([-2.0, -1.0, 0.0, 1.0, 2.0]) ** 2
    f = Qm[None, :] + a[:, None] * R[:, 0][None, :] + b[:, None] * R[:, 4][None, :]
    val, der = oracle.tangential_vec(f, mode, 1, Qm)
    sa = oracle.tangential(a, mode)
    sb = oracle.tangential(b, mode)
    cv = (L @ (val - Qm[None, :]).T).T
    cd = (L @ der.T).T
    assert np.abs(cv[:, 1:4]).max() <= 1e-13 and np.abs(cd[:, 1:4]).max() <= 1e-13
    assert np.allclose(cv[:, 0], sa[0], rtol=0, atol=1e-13)
    assert np.allclose(cd[:, 0], sa[1], rtol=0, atol=1e-13)
    assert np.allclose(cv[:, 4], sb[0], rtol=0, atol=1e-13)
    assert np.allclose(cd[:, 4], sb[1], rtol=0, atol=1e-13)


def test_characteristic_scheme_with_linear_weights_equals_conservative():
    n = (7, 6, 8)
    prim = inputs.random_smooth(n, seed=4, amp=0.2)
    Q = oracle.conservative(prim, GAMMA)
    out = []
    for ch in (0, 1):
        s = oracle.Solver(oracle.Config(*n, recon=0, flux=1, tau_num_C=1.0, mu_ref=1e-3,
                                        char_recon=ch))
        s.set_state(Q)
        out.append(s.rhs(1e-3))
    for k in range(2):
        a, b = out[0][k], out[1][k]
        for v in range(5):
            assert np.abs(a[v] - b[v]).max() <= 1e-11 * np.abs(a[v]).max()


def test_characteristic_weno_z_conserves_and_stays_close_on_smooth_data():
    n = (8, 7, 6)
    prim = inputs.random_smooth(n, seed=6, amp=0.1, kmax=1)
    Q = oracle.conservative(prim, GAMMA)
    res = []
    for ch in (0, 1):
        s = oracle.Solver(oracle.Config(*n, recon=2, flux=1, tau_num_C=1.0, mu_ref=1e-3,
                                        char_recon=ch))
        s.set_state(Q)
        s.step(2, 1e-2)
        res.append(s.state())
    # discrete conservation of the totals (every face flux added once, subtracted once)
    tot0, tot1 = Q.sum(axis=(1, 2, 3)), res[1].sum(axis=(1, 2, 3))
    for v in range(5):
        assert abs(tot1[v] - tot0[v]) <= 1e-13 * np.abs(Q[v]).sum()
    # both are fifth-order reconstructions of the same smooth data
    assert 0 < np.abs(res[1] - res[0]).max() <= 1e-3 * np.abs(res[0]).max()
