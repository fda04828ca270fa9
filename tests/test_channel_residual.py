"""Host part of the channel statistics (hgks_channel_compose, Sec. 3.3;
library host arithmetic, no GPU): from plane means, the scalars and the
wall-unit profiles with the total-stress residual.

* The scalars equal the oracle's (oracle/channel.py) on a laminar profile.
* For the laminar Poiseuille profile the total stress is exactly linear (no
  Reynolds stress): the residual vanishes up to the second-order difference
  of the mean profile on the stretched grid.
* A uniform Reynolds stress <u'v'> = s u_tau^2 shifts the residual by
  exactly -s.
* y+ of the first row and U+ follow from the scalars.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle.channel import channel_stats
from paper_2005_08736_gb300 import _lib, inputs
from paper_2005_08736_gb300.solver import Config, total_stress_residual

G = 1.4
ROWS = _lib.CHANNEL_PROFILES[:8]


@pytest.fixture(scope="module")
def lib():
    try:
        return _lib.load()
    except (RuntimeError, OSError) as e:
        pytest.skip(str(e))


def channel_cfg(ny, mu):
    return Config(6, ny, 6, lx=2 * math.pi, ly=2.0, y0=-1.0, lz=math.pi, y_stretch=1, stretch_b=2.0,
                  bc_y=1, T_wall=100 / 1.4, mu_ref=mu, prec=0)


def laminar(ny, Uc=1.0, V=0.0):
    """Conservative state whose rows hold the cell averages of
    U = Uc (1 - y^2) on the stretched grid (uniform in x, z), optional
    uniform V."""
    yf = inputs.channel_faces(ny)
    ubar = Uc * (1.0 - (yf[:-1] ** 2 + yf[:-1] * yf[1:] + yf[1:] ** 2) / 3.0)
    shape = (2, ny, 2)
    U = np.broadcast_to(ubar[None, :, None], shape).copy()
    rho, p = np.ones(shape), np.full(shape, 70.0)
    Vf = np.full(shape, V)
    cons = np.stack([rho, rho * U, rho * Vf, np.zeros(shape), p / (G - 1) + 0.5 * (U * U + Vf * Vf)])
    return cons, np.diff(yf)


def compose(lib, cfg, prof: dict):
    means = np.ascontiguousarray(np.stack([prof[k] for k in ROWS]))
    out = _lib.HgksChannel()
    rows = np.empty((len(_lib.CHANNEL_PROFILES), cfg.ny))
    pd = ctypes.POINTER(ctypes.c_double)
    c = cfg.c_struct()
    _lib.check(lib.hgks_channel_compose(ctypes.byref(c), means.ctypes.data_as(pd),
                                        rows.ctypes.data_as(pd), ctypes.byref(out)))
    st = {k: getattr(out, k) for k, _ in _lib.HgksChannel._fields_}
    for name, row in zip(_lib.CHANNEL_PROFILES[8:], rows[8:]):
        st[name] = row
    st["profiles"] = dict(zip(ROWS, rows[:8]))
    return st


def test_scalars_match_the_oracle(lib):
    ny, mu = 48, 1e-3
    cons, dy = laminar(ny)
    ref, prof = channel_stats(cons, dy, -1.0, G, mu)
    st = compose(lib, channel_cfg(ny, mu), prof)
    for k in ("tau_w", "tau_w_lower", "tau_w_upper", "rho_w", "u_tau", "Re_tau", "U_b", "U_c",
              "rho_b", "Re_b", "Re_c", "C_f"):
        assert st[k] == pytest.approx(ref[k], rel=1e-12), k


def test_laminar_total_stress_is_linear(lib):
    ny, mu = 96, 1e-3
    cons, dy = laminar(ny)
    _, prof = channel_stats(cons, dy, -1.0, G, mu)
    yp, res = total_stress_residual(compose(lib, channel_cfg(ny, mu), prof))
    assert len(yp) == ny // 2
    # second-order differences of the cell means on the stretched grid
    assert np.abs(res).max() < 2e-2, np.abs(res).max()
    assert np.abs(res[len(res) // 4:]).max() < 5e-3


def test_reynolds_stress_enters_with_its_sign(lib):
    ny, mu = 64, 1e-3
    cfg = channel_cfg(ny, mu)
    cons, dy = laminar(ny)
    _, prof = channel_stats(cons, dy, -1.0, G, mu)
    st0 = compose(lib, cfg, prof)
    # <UV> - <U><V> = s u_tau^2 with s = -0.25 in every row
    shifted = dict(prof)
    shifted["UV"] = prof["UV"] - 0.25 * st0["u_tau"] ** 2
    st1 = compose(lib, cfg, shifted)
    assert np.allclose(st1["uv_plus"], -0.25, atol=1e-13)
    assert np.allclose(st1["total_stress_residual"] - st0["total_stress_residual"], 0.25, atol=1e-13)


def test_wall_units_follow_the_scalars(lib):
    ny, mu = 40, 2e-3
    cons, dy = laminar(ny, Uc=1.5)
    ref, prof = channel_stats(cons, dy, -1.0, G, mu)
    st = compose(lib, channel_cfg(ny, mu), prof)
    assert st["y"][0] == pytest.approx(-1.0 + 0.5 * dy[0], rel=1e-14)
    assert st["y_plus"][0] == pytest.approx(ref["rho_w"] * ref["u_tau"] * 0.5 * dy[0] / mu, rel=1e-12)
    assert st["y_plus"][-1] == pytest.approx(st["y_plus"][0], rel=1e-12)  # symmetric grid
    assert np.allclose(st["U_plus"], prof["U"] / ref["u_tau"], rtol=1e-13)


def test_compose_needs_walls(lib):
    cfg = Config(8, 8, 8, prec=0)
    means = np.ones((8, 8))
    out = _lib.HgksChannel()
    pd = ctypes.POINTER(ctypes.c_double)
    c = cfg.c_struct()
    st = lib.hgks_channel_compose(ctypes.byref(c), means.ctypes.data_as(pd), None, ctypes.byref(out))
    assert st == _lib.HGKS_E_UNSUPPORTED
