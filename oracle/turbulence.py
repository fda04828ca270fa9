"""Oracle of the turbulence statistics of Sec. 3.1 and Sec. 3.4.

TEST INFRASTRUCTURE ONLY: imported by tests/ and by bench.py's reference leg,
never by the product path.  Plain numpy, FP64, periodic uniform grids; it
shares nothing with the CUDA path.

Definitions (Cao, Pan & Xu, arXiv:2005.08736):
  Sec. 3.1: volume-averaged kinetic energy E_k and enstrophy zeta (both scaled
    by 1/(rho0 Omega)); eps(zeta) = 2 mu zeta / rho0; eps(E_k) = -dE_k/dt by
    second-order differences of an E_k history and the numerical dissipation
    eps_num = eps(E_k) - (eps1 + eps2 + eps3); the three Navier-Stokes
    dissipation contributions
    eps1 = 2 mu/rho0 <S^d : S^d>, eps2 = mu_b/rho0 <theta^2>,
    eps3 = -1/rho0 <p theta>, with mu_b = 2N/(3(N+3)) mu and every spatial
    derivative taken by the sixth-order central difference.
  Sec. 3.4: rho_rms, K = 1/2 <rho U.U>, skewness S_u and flatness F_u of the
    velocity slopes d_i U_i, solenoidal dissipation eps_s = <mu omega.omega>,
    dilatational dissipation eps_d = 4/3 <mu theta^2>, pressure dilatation
    <p theta>.
<.> is the volume average over the domain.

Readings: mu is the local viscosity mu(T) of the configured law, kept inside
the averages (the paper's cases with a constant mu are unaffected); S_u and
F_u are the means over the three axes of the per-axis ratios (the printed sum
lacks the 1/3 of an average), and an axis whose <(d_i U_i)^2> is zero is left
out of the mean; the statistics use the full velocity (the mean flow of the
periodic cases is zero).
"""
from __future__ import annotations

import numpy as np

KEYS = ("Ek", "K", "zeta", "eps1", "eps2", "eps3", "rho_mean", "rho_rms", "u_rms",
        "Su", "Fu", "eps_s", "eps_d", "p_theta", "theta_rms", "omega_rms",
        "du2_x", "du2_y", "du2_z", "du3_x", "du3_y", "du3_z", "du4_x", "du4_y", "du4_z",
        "eps_zeta")


def d6(f: np.ndarray, axis: int, h: float) -> np.ndarray:
    """Sixth-order central first derivative on a periodic axis of spacing h:
    the derivative at the centre of the degree-6 interpolant of f_{-3..3}."""
    def s(k):
        return np.roll(f, -k, axis=axis) - np.roll(f, k, axis=axis)
    return (45.0 * s(1) - 9.0 * s(2) + s(3)) / (60.0 * h)


def viscosity(T, law: int, mu_ref: float, T_ref: float, exp: float):
    return mu_ref * np.ones_like(T) if law == 0 else mu_ref * (T / T_ref) ** exp


def statistics(cons: np.ndarray, lengths=(2 * np.pi,) * 3, gamma: float = 1.4, rho0: float = 1.0,
               visc_law: int = 0, mu_ref: float = 1.0 / 1600.0, T_ref: float = 1.0,
               visc_exp: float = 0.76) -> dict:
    """Statistics of the conservative state cons[5][nz][ny][nx] (x fastest)."""
    cons = np.asarray(cons, dtype=np.float64)
    _, nz, ny, nx = cons.shape
    h = (lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
    axis = (2, 1, 0)  # array axis of x, y, z
    rho = cons[0]
    U = [cons[1] / rho, cons[2] / rho, cons[3] / rho]
    q2 = U[0] ** 2 + U[1] ** 2 + U[2] ** 2
    p = (gamma - 1.0) * (cons[4] - 0.5 * rho * q2)
    mu = viscosity(p / rho, visc_law, mu_ref, T_ref, visc_exp)
    N = (5.0 - 3.0 * gamma) / (gamma - 1.0)   # internal degrees of freedom
    mu_b = 2.0 * N / (3.0 * (N + 3.0)) * mu

    # G[i][j] = dU_i / dx_j
    G = [[d6(U[i], axis[j], h[j]) for j in range(3)] for i in range(3)]
    theta = G[0][0] + G[1][1] + G[2][2]
    omega = [G[2][1] - G[1][2], G[0][2] - G[2][0], G[1][0] - G[0][1]]
    w2 = omega[0] ** 2 + omega[1] ** 2 + omega[2] ** 2
    SdSd = np.zeros_like(rho)
    for i in range(3):
        for j in range(3):
            s = 0.5 * (G[i][j] + G[j][i]) - (theta / 3.0 if i == j else 0.0)
            SdSd += s * s

    def avg(f):
        return float(np.mean(f))  # uniform cells: the volume average

    out = {}
    out["Ek"] = avg(0.5 * rho * q2) / rho0
    out["K"] = avg(0.5 * rho * q2)
    out["zeta"] = avg(0.5 * rho * w2) / rho0
    out["eps1"] = 2.0 * avg(mu * SdSd) / rho0
    out["eps2"] = avg(mu_b * theta ** 2) / rho0
    out["eps3"] = -avg(p * theta) / rho0
    rm = avg(rho)
    out["rho_mean"] = rm
    out["rho_rms"] = float(np.sqrt(avg((rho - rm) ** 2)))
    out["u_rms"] = float(np.sqrt(avg(q2) / 3.0))
    m2 = [avg(G[i][i] ** 2) for i in range(3)]
    m3 = [avg(G[i][i] ** 3) for i in range(3)]
    m4 = [avg(G[i][i] ** 4) for i in range(3)]
    live = [i for i in range(3) if m2[i] > 0.0]
    out["Su"] = float(np.mean([m3[i] / m2[i] ** 1.5 for i in live])) if live else 0.0
    out["Fu"] = float(np.mean([m4[i] / m2[i] ** 2 for i in live])) if live else 0.0
    out["eps_s"] = avg(mu * w2)
    out["eps_d"] = 4.0 / 3.0 * avg(mu * theta ** 2)
    out["p_theta"] = avg(p * theta)
    out["theta_rms"] = float(np.sqrt(avg(theta ** 2)))
    out["omega_rms"] = float(np.sqrt(avg(w2)))
    for k, m in (("du2", m2), ("du3", m3), ("du4", m4)):
        for i, a in enumerate("xyz"):
            out[f"{k}_{a}"] = m[i]
    # Sec. 3.1: the incompressible-limit dissipation rate eps(zeta) = 2 mu zeta / rho0
    # (mu the configured viscosity mu_ref; the paper's case has a constant mu).
    out["eps_zeta"] = 2.0 * mu_ref * out["zeta"] / rho0
    return out


def dissipation_history(t, stats):
    """Sec. 3.1 from a time history of statistics (`stats[i]` of the state at
    time t[i]): eps(E_k) = -dE_k/dt by second-order differences of the E_k
    samples (numpy's gradient with second-order one-sided ends; the times may
    be unevenly spaced), and the numerical dissipation
    eps_num = eps(E_k) - (eps1 + eps2 + eps3).  Returns (eps_Ek, eps_num)."""
    t = np.asarray(t, dtype=np.float64)
    ek = np.array([s["Ek"] for s in stats])
    eps_ek = -np.gradient(ek, t, edge_order=2)
    phys = np.array([s["eps1"] + s["eps2"] + s["eps3"] for s in stats])
    return eps_ek, eps_ek - phys
