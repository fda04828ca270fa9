"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds problem set-up only (initial fields of the paper's test
cases and of the convergence test); it contains none of the scheme's
arithmetic.  Every generator returns FP64 numpy arrays of primitive variables
(rho, u, v, w, p) laid out as [5][nz][ny][nx] (x fastest), sampled at cell
centres, unless stated otherwise.

Workloads (Cao, Pan & Xu, arXiv:2005.08736):
  * Taylor-Green vortex, Sec. 3.1.
  * Decaying compressible isotropic turbulence, Sec. 3.4, Eq. (9)-(10).
  * Turbulent channel flow, Sec. 3.3 (tanh-stretched y, laminar profile + noise).
  * Advected density wave: an exact Euler solution used for convergence tests.
"""
from __future__ import annotations

import math

import numpy as np


def centres(n: int, length: float, origin: float = 0.0) -> np.ndarray:
    """Cell centres of a uniform grid of n cells on [origin, origin + length]."""
    return origin + (np.arange(n) + 0.5) * (length / n)


def channel_faces(ny: int, b: float = 2.0) -> np.ndarray:
    """Face positions y_j, j = 0..ny, of the tanh mapping of Sec. 3.3:
    y = tanh(b (eta / (1.5 pi) - 1)) / tanh(b), eta uniform on [0, 3 pi]."""
    eta = 3.0 * math.pi * np.arange(ny + 1) / ny
    return np.tanh(b * (eta / (1.5 * math.pi) - 1.0)) / math.tanh(b)


def taylor_green(n: int, mach: float = 0.1, V0: float = 1.0, rho0: float = 1.0,
                 gamma: float = 1.4, uniform_T: bool = False) -> np.ndarray:
    """Taylor-Green vortex on the periodic box [0, 2 pi]^3 (Sec. 3.1, L = 1).

    u = V0 sin x cos y cos z, v = -V0 cos x sin y cos z, w = 0,
    p = p0 + rho0 V0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2), p0 = rho0 c0^2 / gamma,
    c0 = V0 / Ma.  rho = rho0 by default; uniform_T=True takes rho = p / T0
    with T0 = p0 / rho0 instead.
    """
    x = centres(n, 2 * math.pi)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    c0 = V0 / mach
    p0 = rho0 * c0 * c0 / gamma
    u = V0 * np.sin(x3) * np.cos(y3) * np.cos(z3)
    v = -V0 * np.cos(x3) * np.sin(y3) * np.cos(z3)
    w = np.zeros_like(u)
    p = p0 + rho0 * V0 * V0 / 16.0 * (np.cos(2 * x3) + np.cos(2 * y3)) * (np.cos(2 * z3) + 2.0)
    rho = p / (p0 / rho0) if uniform_T else np.full_like(u, rho0)
    return np.stack([rho, u, v, w, p])


def taylor_green_reference(mach: float = 0.1, V0: float = 1.0, rho0: float = 1.0,
                           gamma: float = 1.4):
    """Reference state (rho, (u, v, w), p) of the Taylor-Green set-up."""
    c0 = V0 / mach
    return rho0, (0.0, 0.0, 0.0), rho0 * c0 * c0 / gamma


def density_wave_cons(n: int, amp: float = 0.2, gamma: float = 1.4, t: float = 0.0,
                      U: float = 1.0, p: float = 1.0) -> np.ndarray:
    """Exact cell averages of the conservative variables of the advected wave
    rho = 1 + amp sin(x + y + z - 3 U t), u = v = w = U, p const, on [0, 2 pi]^3.

    The cell average of sin(x + y + z) over a cube of side h centred at c is
    sin(c_x + c_y + c_z) (sin(h/2) / (h/2))^3.
    """
    h = 2 * math.pi / n
    x = centres(n, 2 * math.pi)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    s = (math.sin(h / 2) / (h / 2)) ** 3
    rho = 1.0 + amp * s * np.sin(x3 + y3 + z3 - 3 * U * t)
    E = p / (gamma - 1.0) + 1.5 * U * U * rho
    return np.stack([rho, U * rho, U * rho, U * rho, E])


def random_smooth(n: tuple[int, int, int], seed: int, amp: float = 0.05,
                  rho0: float = 1.0, p0: float = 1.0, kmax: int = 3) -> np.ndarray:
    """A seeded smooth periodic primitive field: a few random low Fourier modes
    of relative amplitude `amp` around (rho0, 0, 0, 0, p0); shape (nx, ny, nz)."""
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed))
    x = 2 * math.pi * (np.arange(nx) + 0.5) / nx
    y = 2 * math.pi * (np.arange(ny) + 0.5) / ny
    z = 2 * math.pi * (np.arange(nz) + 0.5) / nz
    z3, y3, x3 = np.meshgrid(z, y, x, indexing="ij")
    out = []
    for var, base in enumerate((rho0, 0.0, 0.0, 0.0, p0)):
        f = np.zeros_like(x3)
        for _ in range(4):
            k = rng.integers(-kmax, kmax + 1, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1)
            f += a * np.sin(k[0] * x3 + k[1] * y3 + k[2] * z3 + ph)
        scale = base if base != 0.0 else 1.0
        out.append(base + amp * scale * f / 4.0)
    return np.stack(out)


def isotropic_constants(k0: float = 8.0, A0: float = 1.3e-4, re_lambda: float = 72.0,
                        mach_t: float = 0.5, gamma: float = 1.4, rho0: float = 1.0) -> dict:
    """Initial constants of the isotropic case (Sec. 3.4, Eq. (10) and the
    Re_lambda / Ma_t definitions): K0, u_rms, tau_to, mu0, c0, T0, p0."""
    K0 = 3.0 * A0 / 64.0 * math.sqrt(2 * math.pi) * k0 ** 5
    u_rms = math.sqrt(2.0 * K0 / 3.0)
    mu0 = (2 * math.pi) ** 0.25 / 4.0 * rho0 * math.sqrt(2 * A0) * k0 ** 1.5 / re_lambda
    c0 = math.sqrt(3.0) * u_rms / mach_t
    T0 = c0 * c0 / gamma
    tau_to = math.sqrt(32.0 / A0) * (2 * math.pi) ** 0.25 * k0 ** -3.5
    return dict(K0=K0, u_rms=u_rms, mu0=mu0, c0=c0, T0=T0, p0=rho0 * T0, tau_to=tau_to)


def isotropic(n: int, seed: int, k0: float = 8.0, A0: float = 1.3e-4, mach_t: float = 0.5,
              gamma: float = 1.4, rho0: float = 1.0) -> np.ndarray:
    """Solenoidal random velocity on [0, 2 pi]^3 with spectrum
    E(k) = A0 k^4 exp(-2 k^2 / k0^2) (Sec. 3.4, Eq. (9)), uniform density and
    temperature.  Recipe: seeded complex Gaussian Fourier modes (numpy PCG64),
    projection onto k-orthogonal modes (mean and Nyquist planes removed), each
    integer shell |k| in
    [m - 1/2, m + 1/2) rescaled to the energy E(m), real part of the inverse
    FFT, and a final rescale to u_rms = sqrt(2 K0 / 3).  T0 = c0^2 / gamma with
    c0 = sqrt(3) u_rms / Ma_t; returns primitive (rho, u, v, w, p)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    kk = np.sqrt(k2)
    uh = [rng.normal(size=kk.shape) + 1j * rng.normal(size=kk.shape) for _ in range(3)]
    safe = np.where(k2 > 0, k2, 1.0)
    div = (kx * uh[0] + ky * uh[1] + kz * uh[2]) / safe
    uh = [uh[0] - kx * div, uh[1] - ky * div, uh[2] - kz * div]
    # Drop the mean and the Nyquist planes (k and -k share an index there, so the
    # real part of the inverse transform would not stay solenoidal).
    nyq = (np.abs(kx) == n // 2) | (np.abs(ky) == n // 2) | (np.abs(kz) == n // 2) if n % 2 == 0 \
        else np.zeros_like(k2, dtype=bool)
    for c in range(3):
        uh[c][(k2 == 0) | nyq] = 0.0
    shell = np.floor(kk + 0.5).astype(int)
    energy = 0.5 * sum(np.abs(u) ** 2 for u in uh)
    target = A0 * np.arange(shell.max() + 1) ** 4.0 * np.exp(-2.0 * np.arange(shell.max() + 1) ** 2 / k0 ** 2)
    have = np.bincount(shell.ravel(), weights=energy.ravel(), minlength=len(target))
    scale = np.sqrt(np.where(have > 0, target / np.where(have > 0, have, 1.0), 0.0))
    u = [np.real(np.fft.ifftn(uh[c] * scale[shell])) for c in range(3)]
    cst = isotropic_constants(k0, A0, 72.0, mach_t, gamma, rho0)
    rms = math.sqrt(sum(float((x * x).mean()) for x in u) / 3.0)
    u = [x * (cst["u_rms"] / rms) for x in u]
    rho = np.full_like(u[0], rho0)
    p = np.full_like(u[0], cst["p0"])
    return np.stack([rho, u[0], u[1], u[2], p])


def channel(nx: int, ny: int, nz: int, seed: int, mach: float = 0.1, gamma: float = 1.4,
            b: float = 2.0) -> np.ndarray:
    """Turbulent-channel start of Sec. 3.3 on [0, 2 pi] x [-1, 1] x [0, pi]:
    U = 1.5 (1 - y^2) at the centres of the tanh-stretched y cells, with seeded
    uniform noise of 10 % of the local U on u, v and w; rho = 1 and uniform
    pressure p0 = c0^2 / gamma with c0 = 1 / Ma (unit bulk velocity)."""
    yf = channel_faces(ny, b)
    yc = 0.5 * (yf[1:] + yf[:-1])
    rng = np.random.Generator(np.random.PCG64(seed))
    U = 1.5 * (1.0 - yc ** 2)[None, :, None] * np.ones((nz, ny, nx))
    prim = np.zeros((5, nz, ny, nx))
    prim[0] = 1.0
    prim[1] = U * (1.0 + 0.1 * rng.uniform(-1, 1, U.shape))
    prim[2] = 0.1 * U * rng.uniform(-1, 1, U.shape)
    prim[3] = 0.1 * U * rng.uniform(-1, 1, U.shape)
    prim[4] = (1.0 / mach) ** 2 / gamma
    return prim


def slab(n: tuple[int, int, int], seed: int, axis: int = 0, rho: tuple[float, float] = (1.0, 0.5),
         p: tuple[float, float] = (1.0, 0.4), u_amp: float = 0.1) -> np.ndarray:
    """Piecewise-constant density and pressure with jumps: state 1 (rho[1],
    p[1]) between the planes at a quarter and three quarters of `axis`, state
    0 outside (two periodic contact/pressure jumps, the data on which WENO5's
    nonlinear weights move far from the linear ones), plus a seeded smooth
    velocity (random_smooth's modes, relative amplitude u_amp of unit speed).
    Shape (nx, ny, nz); [0, 2 pi]^3."""
    base = random_smooth(n, seed, amp=u_amp, rho0=1.0, p0=1.0)
    nx, ny, nz = n
    m = (nx, ny, nz)[axis]
    inner = (np.arange(m) >= m // 4) & (np.arange(m) < (3 * m) // 4)
    shape = [1, 1, 1]
    shape[2 - axis] = m
    mask = np.broadcast_to(inner.reshape(shape), (nz, ny, nx))
    out = base.copy()
    out[0] = np.where(mask, rho[1], rho[0])
    out[4] = np.where(mask, p[1], p[0])
    return out


def shear_layer(n: tuple[int, int, int], seed: int, U0: float = 1.0, delta: float = 0.05,
                mach: float = 0.3, amp: float = 0.05, gamma: float = 1.4) -> np.ndarray:
    """Periodic double shear layer on [0, 2 pi]^3: u = U0 tanh((y - pi/2)/delta)
    for y < pi and U0 tanh((3 pi/2 - y)/delta) above (layers thinner than a
    cell at these grids), v and w seeded smooth perturbations of relative
    amplitude `amp` (random_smooth's modes), rho = 1, uniform p = 1/(gamma
    Ma^2) with Ma = mach for U0 = 1.  Shape (nx, ny, nz)."""
    nx, ny, nz = n
    pert = random_smooth(n, seed, amp=amp, rho0=1.0, p0=1.0)
    y = centres(ny, 2 * math.pi)
    u = np.where(y < math.pi, U0 * np.tanh((y - 0.5 * math.pi) / delta),
                 U0 * np.tanh((1.5 * math.pi - y) / delta))
    out = np.empty((5, nz, ny, nx))
    out[0] = 1.0
    out[1] = u[None, :, None]
    out[2] = pert[2] * U0
    out[3] = pert[3] * U0
    out[4] = 1.0 / (gamma * mach * mach)
    return out
