"""Ensembles: one CUDA-graph launch per step for a ragged batch of contexts
gives the same states as stepping each context on its own, bit for bit, in
both forms of the graph -- one batched kernel launch per phase for all
members (instance table), and every member's launches as graph branches."""
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


@pytest.mark.parametrize("batched", [True, False])
@pytest.mark.parametrize("dt", [0.0, 0.02])
@pytest.mark.parametrize("recon,flux,prec", [(2, 1, 1), (0, 0, 0), (1, 1, 0), (2, 0, 1)])
def test_ensemble_equals_members_stepped_alone(recon, flux, prec, dt, batched):
    members = [member(n, s, recon, flux, prec) for s, n in enumerate(SIZES)]
    batch = []
    for cfg, prim in members:
        sim = Simulation(cfg)
        sim.init_primitive(prim)
        batch.append(sim)
    ens = Ensemble(batch, batched=batched)
    ens.step(3, dt)
    ens.step(2, dt, sync=False)  # the members' own streams are ordered after the batch
    for (cfg, prim), sim in zip(members, batch):
        alone = Simulation(cfg)
        alone.init_primitive(prim)
        alone.step(5, dt)
        got, ref = sim.state(), alone.state()
        if batched:
            # the batched kernels are other compilations of the same formulas
            # (fused multiply-adds may be formed differently): rounding-level
            # differences, held to the parity tolerances
            err = rel_linf(got, ref)
            print(f"batched vs alone, prec {prec}: {err:.3e}")
            assert err <= (1e-12 if prec == 0 else 2e-5), err
            assert sim.diagnostics()["t"] == pytest.approx(alone.diagnostics()["t"],
                                                           rel=1e-13 if prec == 0 else 1e-6)
        else:
            assert np.array_equal(got, ref)
            assert sim.diagnostics()["t"] == alone.diagnostics()["t"]
    ens.close()


def rel_linf(a, b):
    scale = [max(np.abs(b[v]).max(), 1e-300) for v in range(5)]
    scale[1:4] = [max(scale[1:4])] * 3
    return max(np.abs(a[v] - b[v]).max() / scale[v] for v in range(5))


@pytest.mark.parametrize("variant", [0, 3])
def test_batched_ensemble_of_walled_channels_and_tile_variants(variant):
    """Batched launches with walls, the stretched grid, the constant force
    and the packed FP32 tile; each member stepped alone as the reference."""
    sizes = [(20, 16, 12), (16, 24, 10), (24, 12, 14)]

    def cfg_of(n):
        return Config(*n, lx=2 * np.pi, ly=2.0, y0=-1.0, lz=np.pi, y_stretch=1, stretch_b=2.0, bc_y=1,
                      T_wall=100 / 1.4, mu_ref=0.0541 / 180, force_x=2.93e-3, prec=1, recon=0, flux=0)
    sims = []
    for k, n in enumerate(sizes):
        sim = Simulation(cfg_of(n))
        sim._call(sim.lib.hgks_set_sweep_shape(sim.h, variant, 0))
        sim.init_primitive(inputs.channel(*n, seed=k))
        sims.append(sim)
    ens = Ensemble(sims, batched=True)
    ens.step(3)
    for k, (n, sim) in enumerate(zip(sizes, sims)):
        alone = Simulation(cfg_of(n))
        alone._call(alone.lib.hgks_set_sweep_shape(alone.h, variant, 0))
        alone.init_primitive(inputs.channel(*n, seed=k))
        alone.step(3)
        err = rel_linf(sim.state(), alone.state())
        print(f"batched channel vs alone, variant {variant}: {err:.3e}")
        assert err <= 2e-5, err
    ens.close()


def test_batched_form_needs_one_scheme():
    from paper_2005_08736_gb300._lib import HGKS_E_UNSUPPORTED, HgksError
    a = Simulation(Config(8, 8, 8, prec=0, recon=0, flux=0))
    b = Simulation(Config(8, 8, 8, prec=0, recon=2, flux=1, tau_num_C=1.0))
    with pytest.raises(HgksError) as e:
        Ensemble([a, b], batched=True)
    assert e.value.status == HGKS_E_UNSUPPORTED
    Ensemble([a, b]).close()  # the graph branches serve any members


def test_ensemble_rejects_a_shared_stream():
    from paper_2005_08736_gb300._lib import HgksError
    s = torch.cuda.Stream()
    a = Simulation(Config(8, 8, 8, prec=0), stream=s)
    b = Simulation(Config(8, 8, 8, prec=0), stream=s)
    with pytest.raises(HgksError):
        Ensemble([a, b])
