"""The kinetic-energy functional on the device (hgks_kinetic_energy, through
the C ABI): E_k of Sec. 3.1 and its gradient dE_k/dQ, the seed of the
adjoint for a final kinetic-energy functional.

* The Taylor-Green start has E_k = 1/8 exactly (cell-centre samples of
  sin^2 cos^2 cos^2 average to 1/8 per component on a periodic grid).
* On the stretched, walled channel grid: against the sum over the oracle's
  state with the oracle's cell volumes.
* The gradient against central differences of the value, and through
  torch.autograd (solver.kinetic_energy).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300.solver import Config, Simulation, kinetic_energy, taylor_green_config  # noqa: E402


def channel_cfg(n):
    return Config(*n, lx=2 * math.pi, ly=2.0, y0=-1.0, lz=math.pi, y_stretch=1, stretch_b=2.0, bc_y=1,
                  T_wall=100 / 1.4, mu_ref=0.0541 / 180, force_x=2.93e-3, prec=0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_taylor_green_start_has_one_eighth(prec):
    cfg = taylor_green_config(16, prec)
    sim = Simulation(cfg)
    q = torch.from_numpy(oracle.conservative(inputs.taylor_green(16), 1.4)).cuda()
    assert sim.kinetic_energy(q) == pytest.approx(0.125, rel=1e-13)
    sim.close()


def test_channel_value_matches_the_oracle_sum():
    n = (12, 16, 10)
    cfg = channel_cfg(n)
    prim = inputs.channel(*n, seed=2)
    Q = oracle.conservative(prim, cfg.gamma)
    o = oracle.Solver(oracle.Config(*n, lx=cfg.lx, ly=2.0, y0=-1.0, lz=cfg.lz, y_stretch=1,
                                    stretch_b=2.0, bc_y=1))
    wx, wy, wz = (o.widths(d) for d in range(3))
    vol = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    ref = (0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0] * vol).sum() / (cfg.lx * cfg.ly * cfg.lz)
    sim = Simulation(cfg)
    got = sim.kinetic_energy(torch.from_numpy(Q).cuda())
    sim.close()
    assert got == pytest.approx(ref, rel=1e-13)


def test_gradient_matches_central_differences_and_autograd():
    n = (10, 9, 8)
    cfg = Config(*n, prec=0, p_ref=1.0)
    Q = torch.from_numpy(oracle.conservative(inputs.random_smooth(n, seed=3, amp=0.3), 1.4)).cuda()
    sim = Simulation(cfg)
    grad = torch.empty_like(Q)
    sim.kinetic_energy(Q, grad)
    assert bool((grad[4] == 0).all())
    gen = torch.Generator(device="cuda").manual_seed(4)
    for _ in range(3):
        v = torch.randn(Q.shape, dtype=torch.float64, device="cuda", generator=gen)
        h = 1e-6
        fd = (sim.kinetic_energy((Q + h * v).contiguous()) -
              sim.kinetic_energy((Q - h * v).contiguous())) / (2 * h)
        ad = float((grad * v).sum())
        assert ad == pytest.approx(fd, rel=1e-7)
    x = Q.clone().requires_grad_(True)
    J = kinetic_energy(x, sim)
    (g,) = torch.autograd.grad(2.0 * J, x)
    assert torch.allclose(g, 2.0 * grad, rtol=0, atol=0)
    sim.close()
