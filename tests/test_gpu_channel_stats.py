"""Channel mean-flow statistics of the CUDA path (hgks_channel_stats, through
the C ABI) against the FP64 oracle's (oracle/channel.py), on a noisy
stretched channel (walls, Sec. 3.3) after two steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.channel import channel_stats  # noqa: E402
from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300._lib import HGKS_E_UNSUPPORTED, HgksError  # noqa: E402
from paper_2005_08736_gb300.solver import Config, Simulation  # noqa: E402

KEYS = ["tau_w", "tau_w_lower", "tau_w_upper", "rho_w", "u_tau", "Re_tau", "U_b", "U_c", "rho_b",
        "Re_b", "Re_c", "C_f"]


def channel_cfg(n, prec):
    return Config(*n, lx=2 * np.pi, ly=2.0, y0=-1.0, lz=np.pi, y_stretch=1, stretch_b=2.0, bc_y=1,
                  T_wall=100 / 1.4, mu_ref=0.0541 / 180, force_x=2.93e-3, prec=prec, recon=0, flux=0)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_channel_statistics_match_oracle(prec, tol):
    n = (24, 32, 12)
    cfg = channel_cfg(n, prec)
    sim = Simulation(cfg)
    sim.init_primitive(inputs.channel(*n, 0))
    sim.step(2)
    got = sim.channel_stats()
    state = sim.state()
    sim.close()
    dy = np.diff(inputs.channel_faces(n[1]))
    ref, prof = channel_stats(state, dy, -1.0, cfg.gamma, cfg.mu_ref)
    for k in KEYS:
        assert got[k] == pytest.approx(ref[k], rel=tol, abs=1e-300), k
    for name, v in prof.items():
        scale = max(np.abs(v).max(), 1e-30)
        assert np.abs(got["profiles"][name] - v).max() <= tol * scale, name
    # wall units: y+ of the first row and U+ consistent with the scalars
    assert got["y_plus"][0] == pytest.approx(
        ref["rho_w"] * ref["u_tau"] * 0.5 * dy[0] / ref["mu_w"], rel=10 * tol)
    assert np.allclose(got["U_plus"], prof["U"] / ref["u_tau"], rtol=10 * tol, atol=0)
    uvp = (prof["UV"] - prof["U"] * prof["V"]) / ref["u_tau"] ** 2
    assert np.abs(got["uv_plus"] - uvp).max() <= 10 * tol * max(np.abs(uvp).max(), 1.0)
    assert np.isfinite(got["total_stress_residual"]).all() and len(got["dUp_dYp"]) == n[1]


def test_channel_statistics_need_walls():
    cfg = Config(8, 8, 8, prec=0)
    sim = Simulation(cfg)
    with pytest.raises(HgksError) as e:
        sim.channel_stats()
    sim.close()
    assert e.value.status == HGKS_E_UNSUPPORTED
