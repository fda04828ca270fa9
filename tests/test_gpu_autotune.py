"""The tile autotuner: every sweep launch shape gives the same step (bitwise
for the march length; to FP32 rounding for the tile variants, whose threads
sum the four Gauss points of a face in another order, or evaluate two points
as the halves of packed FP32 pairs), and the tuner's choice is cached per
configuration."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2005_08736_gb300 import inputs  # noqa: E402
from paper_2005_08736_gb300.solver import Simulation, taylor_green_config  # noqa: E402


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("chunk", [0, 8, 12, 64])
def test_every_launch_shape_gives_the_same_step(variant, chunk):
    n = (40, 20, 17)
    cfg = taylor_green_config(8, "fp32")
    cfg.nx, cfg.ny, cfg.nz = n
    prim = inputs.random_smooth(n, seed=4, amp=0.1, p0=100 / 1.4)
    ref = Simulation(cfg)
    ref.init_primitive(prim)
    ref.step(2)
    sim = Simulation(cfg)
    sim.init_primitive(prim)
    sim._call(sim.lib.hgks_set_sweep_shape(sim.h, variant, chunk))
    sim.step(2)
    a, b = sim.state(), ref.state()
    if variant == 0:
        assert np.array_equal(a, b)
    else:
        # The compatibility state Q0 - Q_ref = (dQl + dQr)/2 + (S_l - S_r)/2
        # cancels half-space moments of size rho sqrt(2 theta / pi) (~7 here),
        # so a reordering of its FP32 operations moves the momentum by a few
        # 1e-7 absolute after two steps: 4e-6 of the range.
        for v in range(5):
            assert np.abs(a[v] - b[v]).max() <= 4e-6 * np.abs(b[v]).max()


def test_autotune_keeps_the_state_and_caches_its_choice(tmp_path):
    cfg = taylor_green_config(32, "fp32")
    sim = Simulation(cfg)
    sim.init_primitive(inputs.taylor_green(32))
    before = sim.state()
    rec = sim.autotune(cache=str(tmp_path / "tune.json"))
    assert not rec["cached"] and rec["variant"] in (0, 1, 2, 3) and rec["sweep_ms"] > 0
    assert np.array_equal(sim.state(), before)
    table = json.load(open(tmp_path / "tune.json"))
    assert len(table) == 1
    again = Simulation(cfg)
    again.init_primitive(inputs.taylor_green(32))
    rec2 = again.autotune(cache=str(tmp_path / "tune.json"))
    assert rec2["cached"] and rec2["variant"] == rec["variant"]
    sim.step(3)
    again.step(3)
    assert np.array_equal(sim.state(), again.state())


def test_packed_and_scalar_tiles_agree_on_a_rough_field():
    # The packed tile forms the compatibility state's midpoint rule (small
    # jumps) in pair arithmetic with its tangent written out by the chain
    # rule; the scalar tiles take the same tangent from a dual-number pass of
    # the sign moments.  On a rough field, where the jumps between the two
    # reconstructed states are large enough for a wrong term to show, the two
    # agree to FP32 rounding.
    n = (40, 20, 17)
    cfg = taylor_green_config(8, "fp32")
    cfg.nx, cfg.ny, cfg.nz = n
    prim = inputs.random_smooth(n, seed=9, amp=0.2, kmax=4, p0=100 / 1.4)
    out = []
    for variant in (1, 3):
        sim = Simulation(cfg)
        sim.init_primitive(prim)
        sim._call(sim.lib.hgks_set_sweep_shape(sim.h, variant, 0))
        sim.step(2, 2e-3)
        out.append(sim.state())
        sim.close()
    a, b = out
    for v in range(5):
        assert np.abs(a[v] - b[v]).max() <= 1e-6 * np.abs(b[v]).max(), v
