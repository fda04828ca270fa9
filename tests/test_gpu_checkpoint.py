"""Checkpoint and resume (state through hgks_get_state /
hgks_init_conservative, time and step counter through hgks_set_time): a run
resumed from a checkpoint continues as the uninterrupted run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300.solver import Simulation, taylor_green_config  # noqa: E402


# The state is stored as its deviation from the reference state; the FP64
# round trip Q_ref + q -> Q -> Q - Q_ref rounds in the last bit of the total
# energy (~178 here), which the next steps carry into every variable.
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_resumed_run_continues_the_run(tmp_path, prec, tol):
    cfg = taylor_green_config(16, prec, "weno-z", "full")
    a = Simulation(cfg)
    a.init_primitive(inputs.taylor_green(16))
    a.step(3)
    path = str(tmp_path / "ck.npz")
    a.save_checkpoint(path)
    t_a = a.step(2)
    sa, da = a.state(), a.diagnostics()
    a.close()
    b = Simulation(cfg)
    b.load_checkpoint(path)
    t_b = b.step(2)
    sb, db = b.state(), b.diagnostics()
    b.close()
    assert db["step"] == da["step"] == 5
    assert t_b == pytest.approx(t_a, rel=1e-15)
    mom = np.abs(sa[1:4]).max()  # the momentum components share one scale (rho W starts at 0)
    scale = [np.abs(sa[0]).max(), mom, mom, mom, np.abs(sa[4]).max()]
    for v in range(5):
        assert np.abs(sa[v] - sb[v]).max() <= tol * scale[v], v
