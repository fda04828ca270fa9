"""Host logic of the differentiable step window (CPU only).

solver.StepWindow keeps a checkpoint every `every` steps in the forward pass
and, in the backward pass, recomputes each window from its checkpoint and
applies the adjoint steps in reverse, each at the state it belongs to.  Here
it drives a stand-in simulator with the same interface whose step is a small
nonlinear map with an exact vector-Jacobian product (torch autograd on the
CPU); the window's gradient must equal autograd through the composed map,
for windows that divide the step count, leave a ragged last window, or hold
every step.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2005_08736_gb300.solver import run_window  # noqa: E402


class MapSim:
    """q -> q + dt sin(M q) on CPU tensors, with the methods StepWindow uses."""

    def __init__(self, shape, seed):
        g = torch.Generator().manual_seed(seed)
        self.shape = shape
        n = int(np.prod(shape))
        self.M = torch.randn(n, n, generator=g, dtype=torch.float64) / math.sqrt(n)
        self.q = None
        self.adjoint_states = []

    def f(self, q, dt):
        return q + dt * torch.sin(self.M @ q.reshape(-1)).reshape(self.shape)

    def init_conservative(self, q):
        self.q = q.detach().clone()

    def state(self, device=False):
        return self.q.clone()

    def step(self, nsteps, dt):
        with torch.no_grad():
            for _ in range(nsteps):
                self.q = self.f(self.q, dt)

    def adjoint_step(self, dt, lam, out):
        self.adjoint_states.append(self.q.clone())
        with torch.enable_grad():  # backward passes run with grad mode off
            q = self.q.detach().requires_grad_(True)
            (g,) = torch.autograd.grad(self.f(q, dt), q, lam)
        out.copy_(g)


@pytest.mark.parametrize("nsteps,every", [(6, 3), (7, 3), (5, 1), (4, 10)])
def test_window_gradient_equals_autograd_of_the_composed_map(nsteps, every):
    shape, dt = (5, 2, 3, 2), 0.3
    sim = MapSim(shape, seed=1)
    g = torch.Generator().manual_seed(2)
    q0 = torch.randn(*shape, generator=g, dtype=torch.float64)
    w = torch.randn(*shape, generator=g, dtype=torch.float64)

    x = q0.clone().requires_grad_(True)
    J = ((w * run_window(x, sim, nsteps, dt, every)).sum()
         + (run_window(x, sim, nsteps, dt, every) ** 2).sum())
    J.backward()

    y = q0.clone().requires_grad_(True)
    z = y
    states = []
    for _ in range(nsteps):
        states.append(z.detach().clone())
        z = sim.f(z, dt)
    ref = (w * z).sum() + (z ** 2).sum()
    ref.backward()
    assert torch.allclose(x.grad, y.grad, rtol=1e-13, atol=1e-13)
    # each adjoint step ran at its own state, last step first (two windows
    # were differentiated, one per use of run_window above)
    per_call = sim.adjoint_states[-nsteps:]
    for n, s in enumerate(reversed(per_call)):
        assert torch.equal(s, states[n])
