"""The total-stress residual of the channel (Sec. 3.3; host logic, CPU):
for the laminar Poiseuille profile the total stress is exactly linear
(no Reynolds stress), so the residual vanishes up to the second-order
difference of the mean profile; a uniform Reynolds stress shifts it by
exactly that stress in wall units."""
import math

import numpy as np

from oracle.channel import channel_stats
from paper_2005_08736_gb300 import inputs
from paper_2005_08736_gb300.solver import total_stress_residual

G = 1.4


def stats_of(ny=96, Uc=1.0, mu=1e-3, uv=0.0):
    yf = inputs.channel_faces(ny)
    dy = np.diff(yf)
    yc = 0.5 * (yf[1:] + yf[:-1])
    ubar = Uc * (1.0 - (yf[:-1] ** 2 + yf[:-1] * yf[1:] + yf[1:] ** 2) / 3.0)
    shape = (2, ny, 2)
    U = np.broadcast_to(ubar[None, :, None], shape).copy()
    rho, p = np.ones(shape), np.full(shape, 70.0)
    cons = np.stack([rho, rho * U, np.zeros(shape), np.zeros(shape), p / (G - 1) + 0.5 * U * U])
    out, prof = channel_stats(cons, dy, -1.0, G, mu)
    st = dict(out)
    st["profiles"] = prof
    st["y"] = yc
    dist = np.minimum(yc + 1.0, 1.0 - yc)
    st["y_plus"] = out["rho_w"] * out["u_tau"] * dist / mu
    st["uv_plus"] = np.full(ny, uv)
    return st


def test_laminar_total_stress_is_linear():
    yp, res = total_stress_residual(stats_of())
    assert len(yp) > 10
    # second-order differences of the cell means on the stretched grid
    assert np.abs(res).max() < 2e-2, np.abs(res).max()
    assert np.abs(res[len(res) // 4:]).max() < 5e-3


def test_reynolds_stress_enters_with_its_sign():
    _, r0 = total_stress_residual(stats_of())
    _, r1 = total_stress_residual(stats_of(uv=-0.25))
    assert np.allclose(r1 - r0, 0.25, atol=1e-14)
