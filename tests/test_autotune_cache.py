"""Host logic of the autotuner's choice cache (CPU only).

Simulation.autotune keys each stored launch-shape choice by the full
configuration: a configuration seen before reuses its stored choice (no
timing run), a new one is timed and added, and the JSON file keeps every
entry.  The library calls are replaced by a stand-in that records them.
"""
import json

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2005_08736_gb300.solver import Simulation, taylor_green_config  # noqa: E402


class StandInLib:
    def __init__(self):
        self.timed, self.applied = 0, []

    def hgks_autotune(self, h, variant, chunk, ms):
        self.timed += 1
        variant._obj.value, chunk._obj.value, ms._obj.value = 3, 16, 1.25
        return 0

    def hgks_set_sweep_shape(self, h, variant, chunk):
        self.applied.append((variant, chunk))
        return 0


def stand_in(cfg, lib):
    sim = object.__new__(Simulation)   # no device context: only the cache logic runs
    sim.lib, sim.h, sim.cfg = lib, None, cfg
    return sim


def test_choices_are_cached_per_configuration(tmp_path):
    path = str(tmp_path / "tune.json")
    lib = StandInLib()
    a = stand_in(taylor_green_config(32, "fp32"), lib)
    r = a.autotune(cache=path)
    assert r == {"variant": 3, "chunk": 16, "sweep_ms": 1.25, "cached": False} and lib.timed == 1
    r = a.autotune(cache=path)
    assert r["cached"] and (r["variant"], r["chunk"]) == (3, 16)
    assert lib.timed == 1 and lib.applied == [(3, 16)]
    b = stand_in(taylor_green_config(48, "fp32"), lib)   # another configuration is timed
    assert not b.autotune(cache=path)["cached"] and lib.timed == 2
    with open(path) as fh:
        table = json.load(fh)
    assert len(table) == 2
    # without a cache file every call times the candidates
    assert not a.autotune()["cached"] and lib.timed == 3


@pytest.mark.parametrize("ly,stretch", [(2.0, 1), (3.0, 0)])
def test_library_cell_widths_match_the_oracle_grid(ly, stretch):
    # hgks_cell_widths (host function of the library, no device work): the
    # y widths the statistics and the kinetic-energy functional use, against
    # the oracle's widths (the tanh mapping spans the channel height 2).
    import oracle
    from paper_2005_08736_gb300 import _lib
    from paper_2005_08736_gb300.solver import Config, cell_widths
    try:
        _lib.load()
    except (RuntimeError, OSError) as e:
        pytest.skip(str(e))
    cfg = Config(8, 12, 8, ly=ly, y0=-0.5 * ly, y_stretch=stretch, stretch_b=2.0, bc_y=1)
    got = cell_widths(cfg, 1)
    o = oracle.Solver(oracle.Config(8, 12, 8, ly=ly, y0=-0.5 * ly, y_stretch=stretch,
                                    stretch_b=2.0, bc_y=1))
    assert got == pytest.approx(o.widths(1), rel=1e-13)
    assert got.sum() == pytest.approx(ly, rel=1e-14)
    assert cell_widths(cfg, 0) == pytest.approx(np.full(8, cfg.lx / 8), rel=1e-15)
