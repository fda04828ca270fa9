"""Ensembles: one CUDA-graph launch per step for a ragged batch of contexts
gives the same states as stepping each context on its own."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300.solver import Config, Ensemble, Simulation  # noqa: E402

SIZES = [(16, 16, 16), (20, 12, 14), (12, 12, 12), (24, 10, 8)]


def member(n, seed, recon, flux, prec):
    cfg = Config(*n, prec=prec, recon=recon, flux=flux, tau_num_C=1.0, mu_ref=2e-3, p_ref=1.0,
                 visc=1, visc_exp=0.76, T_ref=1.0, prandtl=0.7)
    prim = inputs.random_smooth(n, seed=seed, amp=0.1)
    return cfg, prim


@pytest.mark.parametrize("dt", [0.0, 0.02])
@pytest.mark.parametrize("recon,flux,prec", [(2, 1, 1), (0, 0, 0)])
def test_ensemble_equals_members_stepped_alone(recon, flux, prec, dt):
    members = [member(n, s, recon, flux, prec) for s, n in enumerate(SIZES)]
    batch = []
    for cfg, prim in members:
        sim = Simulation(cfg)
        sim.init_primitive(prim)
        batch.append(sim)
    ens = Ensemble(batch)
    ens.step(4, dt)
    for (cfg, prim), sim in zip(members, batch):
        alone = Simulation(cfg)
        alone.init_primitive(prim)
        alone.step(4, dt)
        assert np.array_equal(sim.state(), alone.state())
        assert sim.diagnostics()["t"] == alone.diagnostics()["t"]
    ens.close()


def test_ensemble_rejects_a_shared_stream():
    from paper_2005_08736_gb300._lib import HgksError
    s = torch.cuda.Stream()
    a = Simulation(Config(8, 8, 8, prec=0), stream=s)
    b = Simulation(Config(8, 8, 8, prec=0), stream=s)
    with pytest.raises(HgksError):
        Ensemble([a, b])
