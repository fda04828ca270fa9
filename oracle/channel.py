"""FP64 mean-flow statistics of the wall-bounded channel (Sec. 3.3): plain
numpy from a conservative state.

TEST INFRASTRUCTURE ONLY: only tests/ may import this module; it shares no
code with the CUDA path.

Definitions (Sec. 3.3, with the readings where the paper is silent or garbled):
  plane means over x and z of each y row;
  tau_w = mu(T_wall) d<U>/dn at each wall (the paper writes tau_wall =
  dU/dy|wall; the viscosity makes it a stress), d<U>/dn from the quadratic
  a s + b s^2 (s = distance from the wall, <U> = 0 there) whose averages
  over the two wall-adjacent cells equal theirs;
  u_tau = sqrt(tau_w / rho_w), rho_w the mean of the two wall rows' <rho>;
  Re_tau = rho_w u_tau H / mu_w, H = ly / 2;
  U_b, rho_b: height averages; U_c: <U> at the mid-plane from the cubic whose
  averages over the four cells nearest to it equal theirs;
  nu = mu_w / rho_b, Re_c = U_c H / nu, Re_b = 2 U_b H / nu,
  C_f = tau_w / (rho_b U_b^2 / 2).
"""
from __future__ import annotations

import numpy as np


def _avg_pow(a, b, p):
    """Mean of s^p over [a, b]."""
    return (b ** (p + 1) - a ** (p + 1)) / ((p + 1) * (b - a))


def _wall_slope(w1, w2, u1, u2):
    M = np.array([[_avg_pow(0.0, w1, 1), _avg_pow(0.0, w1, 2)],
                  [_avg_pow(w1, w1 + w2, 1), _avg_pow(w1, w1 + w2, 2)]])
    return np.linalg.solve(M, np.array([u1, u2]))[0]


def channel_stats(cons, dy, y0, gamma, mu_w):
    """cons: conservative FP64 state [5][nz][ny][nx]; dy: the ny cell widths
    in y; y0: the lower wall.  Returns the statistics and the plane means."""
    cons = np.asarray(cons, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    rho = cons[0]
    U, V, W = cons[1] / rho, cons[2] / rho, cons[3] / rho
    p = (gamma - 1.0) * (cons[4] - 0.5 * rho * (U * U + V * V + W * W))
    mean = lambda a: a.mean(axis=(0, 2))  # noqa: E731  (over z and x)
    prof = {"rho": mean(rho), "rhoU": mean(cons[1]), "U": mean(U), "V": mean(V), "W": mean(W),
            "UV": mean(U * V), "UU": mean(U * U), "T": mean(p / rho)}
    ny, ly = len(dy), dy.sum()
    Um, rm = prof["U"], prof["rho"]
    lo = _wall_slope(dy[0], dy[1], Um[0], Um[1])
    hi = _wall_slope(dy[-1], dy[-2], Um[-1], Um[-2])
    out = {"tau_w_lower": mu_w * lo, "tau_w_upper": mu_w * hi}
    out["tau_w"] = 0.5 * (out["tau_w_lower"] + out["tau_w_upper"])
    out["mu_w"] = mu_w
    out["rho_w"] = 0.5 * (rm[0] + rm[-1])
    out["u_tau"] = np.sqrt(out["tau_w"] / out["rho_w"])
    H = 0.5 * ly
    out["Re_tau"] = out["rho_w"] * out["u_tau"] * H / mu_w
    out["U_b"] = (Um * dy).sum() / ly
    out["rho_b"] = (rm * dy).sum() / ly
    faces = y0 + np.concatenate([[0.0], np.cumsum(dy)])
    yc = y0 + H
    centres4 = [0.5 * (faces[j] + faces[j + 4]) for j in range(ny - 3)]
    j0 = int(np.argmin(np.abs(np.array(centres4) - yc)))
    M = np.array([[_avg_pow(faces[j0 + k] - yc, faces[j0 + k + 1] - yc, pw) for pw in range(4)]
                  for k in range(4)])
    out["U_c"] = np.linalg.solve(M, Um[j0:j0 + 4])[0]
    nu = mu_w / out["rho_b"]
    out["Re_c"] = out["U_c"] * H / nu
    out["Re_b"] = out["U_b"] * 2.0 * H / nu
    out["C_f"] = out["tau_w"] / (0.5 * out["rho_b"] * out["U_b"] ** 2)
    return out, prof
