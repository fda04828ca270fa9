"""How the oracle's right-hand side is assembled from its pieces (CPU only).

The pieces - WENO5 end values, the compatibility state, the flux at one
point, the ghost fill of the walls, the stretched widths - have pins of
their own.  This test pins the wiring between them: on a state that varies
only along the stretched, walled y axis, with the full flux and a positive
collision time (so that the left and right states and their slopes enter),
it forms the face fields from the defining conditions of each reading of
Sec. 2.1 (the quadratic through both end values and the cell average for the
normal slopes of the two states, the cubic through four cell averages for
the equilibrium slope), passes them to the point flux and takes the
difference over each cell.  The x and z faces of such a state carry equal
fluxes on both sides of a cell and the tangential reconstruction sees
constant data, so the result must equal the oracle's L and dL/dt.  A slope
paired with the wrong state, a width of the wrong cell or a momentum
component in the wrong slot fails it.
"""
import numpy as np
import pytest

import oracle

GAMMA = 1.4
NY = 12
DT = 1e-3


def quadratic_slope(QL, QR, Qbar, s):
    """d/ds at s of the quadratic on the cell s in [-1/2, 1/2] with the end
    values QL, QR and the average Qbar (per unit cell length)."""
    A = np.array([[1.0, -0.5, 0.25], [1.0, 0.5, 0.25], [1.0, 0.0, 1.0 / 12.0]])
    a, b, c = np.linalg.solve(A, np.stack([QL, QR, Qbar]))
    return b + 2.0 * c * s


def cubic_slope(q4, h):
    """Derivative at x = 0 of the cubic whose averages over [-2h,-h], [-h,0],
    [0,h], [h,2h] are q4[0..3]."""
    edges = np.array([-2.0, -1.0, 0.0, 1.0, 2.0]) * h
    A = np.array([[(edges[i + 1] ** (k + 1) - edges[i] ** (k + 1)) / ((k + 1) * h) for k in range(4)]
                  for i in range(4)])
    return np.linalg.solve(A, np.stack(q4))[1]


def to_local_y(Q):
    """(rho, rho u, rho v, rho w, rho E) -> the frame of a y face:
    normal y, then t1 = z, t2 = x."""
    return np.array([Q[0], Q[2], Q[3], Q[1], Q[4]])


def to_global_y(F):
    return np.array([F[0], F[3], F[1], F[2], F[4]])


@pytest.mark.parametrize("recon", [oracle.RECON_WENO_JS, oracle.RECON_WENO_Z])
def test_rhs_is_the_difference_of_point_fluxes_of_the_face_fields(recon):
    Tw = 71.43
    cfg = oracle.Config(6, NY, 6, ly=2.0, y0=-1.0, y_stretch=1, stretch_b=2.0, bc_y=1, T_wall=Tw,
                        mu_ref=0.02, recon=recon, flux=oracle.FLUX_FULL, tau_num_C=1.0,
                        prandtl=0.72)
    rng = np.random.default_rng(7)
    prof = rng.normal(size=(5, NY))
    y = np.arange(NY) - NY / 2 + 0.5
    prim = np.zeros((5, 6, NY, 6))
    prim[0] = (1.0 + 0.25 * np.sign(y) + 0.05 * prof[0])[None, :, None]   # a jump mid-channel
    prim[1] = (1.0 + 0.3 * prof[1])[None, :, None]
    prim[2] = (0.2 * prof[2])[None, :, None]
    prim[3] = (-0.4 + 0.3 * prof[3])[None, :, None]
    prim[4] = (Tw * (1.0 + 0.1 * prof[4]))[None, :, None]
    s = oracle.Solver(cfg)
    s.set_state(oracle.conservative(prim, GAMMA))
    L, dL = s.rhs(DT)

    col = s.padded()[:, 3, :, 3]                  # padded along y: cell j at j + 3
    w = s.widths(1)
    wp = np.concatenate([w[2::-1], w, w[:-4:-1]])  # ghost widths mirror the interior across each wall
    G = np.zeros((NY + 1, 10))
    for f in range(NY + 1):                        # face f between cells f-1 and f
        qc = np.array([to_local_y(col[:, f + k]) for k in range(6)])   # cells f-3 .. f+2
        QRi, QLi, QLr, QRr = oracle.normal_end_values(qc, recon, 0, GAMMA)
        hl, hr = wp[f + 2], wp[f + 3]
        st = np.zeros((3, 4, 5))
        st[0, 0], st[0, 1] = QRi, quadratic_slope(QLi, QRi, qc[2], 0.5) / hl
        st[1, 0], st[1, 1] = QLr, quadratic_slope(QLr, QRr, qc[3], -0.5) / hr
        st[2, 0] = oracle.compat(QRi, QLr, GAMMA)
        st[2, 1] = cubic_slope(qc[1:5], 0.5 * (hl + hr))
        F, dF = oracle.flux_point(cfg, st, DT)
        G[f, :5], G[f, 5:] = to_global_y(F), to_global_y(dF)
    acc = -G[:-1] / w[:, None] + G[1:] / w[:, None]
    L_exp, dL_exp = -acc[:, :5].T, -acc[:, 5:].T
    assert np.abs(L).max() > 1.0 and np.abs(dL).max() > 1.0
    for k in (0, 5):
        for i in (0, 2):
            assert np.abs(L[:, k, :, i] - L_exp).max() <= 1e-11 * np.abs(L).max()
            assert np.abs(dL[:, k, :, i] - dL_exp).max() <= 1e-11 * np.abs(dL).max()
