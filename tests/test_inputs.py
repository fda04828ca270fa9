"""The seeded input generators (problem set-up of Sec. 3.1, 3.3, 3.4): the
isotropic constants against the paper's printed resolution table, the
isotropic field's divergence, r.m.s. velocity and spectrum, the channel start
and the Taylor-Green field (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from paper_2005_08736_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def test_isotropic_constants_reproduce_the_printed_resolution_table():
    tab = json.load(open(GOLDEN))["isotropic_resolution"]
    n = tab["n"]
    delta = 2 * math.pi / n
    for r in tab["rows"]:
        c = inputs.isotropic_constants(k0=8.0, A0=1.3e-4, re_lambda=72.0, mach_t=r["mach_t"])
        nu0 = c["mu0"]  # rho0 = 1
        omega0 = 15 * 1.3e-4 / 256 * math.sqrt(2 * math.pi) * 8.0 ** 7   # Eq. (10)
        eps0 = 2 * nu0 * omega0
        eta0 = (nu0 ** 3 / eps0) ** 0.25
        lam0 = 3 * c["mu0"] / c["c0"]   # mu0 = rho0 c0 lambda0 / 3
        kmax = math.sqrt(2) * n / 3
        assert kmax * eta0 == pytest.approx(r["kmax_eta0"], abs=1e-3)
        assert delta / eta0 == pytest.approx(r["delta_over_eta0"], abs=1.5e-3)
        assert delta / lam0 == pytest.approx(r["delta_over_lambda0"], abs=1.5e-3)


def test_isotropic_field_is_solenoidal_with_the_requested_rms():
    n, k0 = 32, 4.0
    prim = inputs.isotropic(n, seed=3, k0=k0, mach_t=0.5)
    c = inputs.isotropic_constants(k0=k0, mach_t=0.5)
    u = prim[1:4]
    assert math.sqrt((u ** 2).mean()) == pytest.approx(c["u_rms"], rel=1e-12)
    k = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    uh = [np.fft.fftn(x) for x in u]
    div = kx * uh[0] + ky * uh[1] + kz * uh[2]
    assert np.abs(div).max() <= 1e-9 * max(np.abs(h).max() for h in uh)
    assert np.allclose(prim[0], 1.0) and np.allclose(prim[4], c["p0"])
    # The energy spectrum peaks near k0 (Eq. (9): E ~ k^4 exp(-2 k^2 / k0^2)).
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    shell = np.floor(kk + 0.5).astype(int)
    e = np.bincount(shell.ravel(), weights=0.5 * sum(np.abs(h) ** 2 for h in uh).ravel())
    assert abs(int(np.argmax(e)) - k0) <= 1


def test_isotropic_field_depends_only_on_the_seed():
    a = inputs.isotropic(16, seed=5, k0=4.0)
    b = inputs.isotropic(16, seed=5, k0=4.0)
    c = inputs.isotropic(16, seed=6, k0=4.0)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_channel_start():
    prim = inputs.channel(8, 16, 6, seed=0)
    yf = inputs.channel_faces(16)
    yc = 0.5 * (yf[1:] + yf[:-1])
    U = 1.5 * (1 - yc ** 2)
    assert np.all(np.abs(prim[1] / U[None, :, None] - 1) <= 0.1 + 1e-12)
    assert np.all(np.abs(prim[2]) <= 0.1 * U[None, :, None] + 1e-12)
    assert np.allclose(prim[4], 100 / 1.4)
    assert yf[0] == pytest.approx(-1) and yf[-1] == pytest.approx(1)


def test_taylor_green_initial_kinetic_energy_and_divergence():
    prim = inputs.taylor_green(32)
    ek = 0.5 * (prim[0] * (prim[1] ** 2 + prim[2] ** 2 + prim[3] ** 2)).mean()
    assert ek == pytest.approx(0.125, rel=1e-12)   # <sin^2 cos^2 cos^2> terms, Sec. 3.1
    assert prim[4].min() > 0 and np.allclose(prim[0], 1.0)


def test_config_presets_carry_the_papers_constants():
    import math
    from paper_2005_08736_gb300.solver import channel_config, isotropic_config
    ch = channel_config()
    assert (ch.nx, ch.ny, ch.nz) == (128, 128, 96)
    assert ch.mu_ref == pytest.approx(0.0541 / 180) and ch.force_x == pytest.approx(2.93e-3)
    assert ch.bc_y == 1 and ch.y_stretch == 1 and ch.ly == 2.0 and ch.lx == pytest.approx(2 * math.pi)
    assert ch.T_wall == pytest.approx(100 / 1.4)  # c0 = 10 with U_b = 1 (Ma 0.1)
    iso = isotropic_config(64, k0=4.0)
    c = inputs.isotropic_constants(k0=4.0, mach_t=0.5)
    assert iso.mu_ref == pytest.approx(c["mu0"]) and iso.p_ref == pytest.approx(c["p0"])
    assert iso.visc == 1 and iso.visc_exp == 0.76 and iso.prandtl == 0.7
    assert iso.recon == 2 and iso.flux == 1 and iso.tau_num_C == 1.0
