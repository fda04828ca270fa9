"""The oracle's operation-counting build (CPU only): the same source compiled
with a tallying scalar type reproduces the plain oracle bit for bit, and its
tallies behave as operation counts (positive, more work for WENO-Z + the full
flux than for linear weights + the smooth flux, and a per-cell count that
falls as the grid grows, because the face fields carry two tangential ghost
rows)."""
import numpy as np

import oracle
from paper_2005_08736_gb300 import inputs


def run(n, recon, flux):
    cfg = oracle.Config(n, n, n, recon=recon, flux=flux, tau_num_C=1.0 if flux else 0.0)
    q = oracle.conservative(inputs.taylor_green(n), 1.4)
    state, tally = oracle.count_step(cfg, q, 1, 1e-3)
    s = oracle.Solver(cfg)
    s.set_state(q)
    s.step(1, 1e-3)
    return state, s.state(), tally


def flops(t):
    return t["add"] + t["mul"] + t["div"]


def test_counting_build_reproduces_the_plain_oracle():
    for recon, flux in ((0, 0), (2, 1)):
        counted, plain, tally = run(8, recon, flux)
        assert np.array_equal(counted, plain)
        assert all(v >= 0 for v in tally.values()) and flops(tally) > 0


def test_counts_order_and_grid_dependence():
    _, _, smooth8 = run(8, 0, 0)
    _, _, full8 = run(8, 2, 1)
    _, _, smooth12 = run(12, 0, 0)
    assert flops(full8) > 2 * flops(smooth8)
    assert full8["erfc"] > smooth8["erfc"] > 0  # half-space moments of l, r (and Q0)
    per8, per12 = flops(smooth8) / 8 ** 3, flops(smooth12) / 12 ** 3
    assert per12 < per8 < 1.2 * per12
