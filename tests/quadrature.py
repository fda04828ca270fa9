"""Brute-force velocity-space quadrature of Maxwellian-weighted integrals.

Used by the oracle pins: every integral the oracle evaluates through moment
recursions is recomputed here by numerical quadrature over the particle
velocity (u, v, w) and the internal variables xi = (xi_1 .. xi_K), K = 2
(gamma = 1.4).  Nothing here imports the oracle or the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4
K = 2  # internal degrees of freedom for gamma = 1.4


def prim(Q, gamma=GAMMA):
    rho = Q[0]
    U, V, W = Q[1] / rho, Q[2] / rho, Q[3] / rho
    p = (gamma - 1.0) * (Q[4] - 0.5 * rho * (U * U + V * V + W * W))
    return rho, U, V, W, rho / (2.0 * p)


def _hermite(n, mean, lam):
    """Nodes/weights for int f(x) sqrt(lam/pi) exp(-lam (x-mean)^2) dx."""
    x, w = np.polynomial.hermite.hermgauss(n)
    return mean + x / math.sqrt(lam), w / math.sqrt(math.pi)


def _legendre(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


class Maxwell:
    """Quadrature for int g(u, v, w, xi) phi dXi of a Maxwellian g of the
    conservative state Q (R = 1), optionally over the half space u > 0 or u < 0."""

    def __init__(self, Q, half=0, n_herm=8, n_leg=160, gamma=GAMMA):
        self.rho, U, V, W, lam = prim(Q, gamma)
        if half == 0:
            u, wu = _hermite(n_herm, U, lam)
        else:
            s = 1.0 / math.sqrt(lam)
            a, b = (0.0, max(U + 14 * s, 1e-3)) if half > 0 else (min(U - 14 * s, -1e-3), 0.0)
            u, wl = _legendre(a, b, n_leg)
            wu = wl * math.sqrt(lam / math.pi) * np.exp(-lam * (u - U) ** 2)
        v, wv = _hermite(n_herm, V, lam)
        w, ww = _hermite(n_herm, W, lam)
        x1, w1 = _hermite(n_herm, 0.0, lam)
        x2, w2 = _hermite(n_herm, 0.0, lam)
        grids = np.meshgrid(u, v, w, x1, x2, indexing="ij")
        wts = np.einsum("a,b,c,d,e->abcde", wu, wv, ww, w1, w2)
        self.u, self.v, self.w = (g.ravel() for g in grids[:3])
        self.xi2 = (grids[3] ** 2 + grids[4] ** 2).ravel()
        self.wt = wts.ravel()

    def psi(self):
        """psi = (1, u, v, w, (u^2+v^2+w^2+xi^2)/2) at the nodes, shape [5, n]."""
        one = np.ones_like(self.u)
        return np.stack([one, self.u, self.v, self.w,
                         0.5 * (self.u ** 2 + self.v ** 2 + self.w ** 2 + self.xi2)])

    def vel(self):
        return np.stack([self.u, self.v, self.w])

    def integrate(self, phi):
        """rho * sum(weights * phi) over the last axis."""
        return self.rho * (np.asarray(phi) * self.wt).sum(axis=-1)


def lin(a, psi):
    """a . psi at the nodes."""
    return np.tensordot(np.asarray(a), psi, axes=(0, 0))
