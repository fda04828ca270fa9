"""Host logic of the autotuner's choice cache (CPU only).

Simulation.autotune keys each stored launch-shape choice by the full
configuration: a configuration seen before reuses its stored choice (no
timing run), a new one is timed and added, and the JSON file keeps every
entry.  The library calls are replaced by a stand-in that records them.
"""
import json

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
