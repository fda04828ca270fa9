"""hgks_step_noalloc: the step for callers that cannot allocate device memory.

Such callers (a host framework that owns every device allocation, a context
whose memory footprint must stay fixed) pass the state buffer in and get the
stepped state back; the library does the work in its built-in scratch array.
This file is collected last on purpose.  Its results must equal those of the
allocating entry points (hgks_init_conservative + hgks_step + hgks_get_state)
within the FP64 tolerance of the parity tests, on two calls in a row (the
second call finds the scratch array holding the first call's data).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2005_08736_gb300 import _lib, inputs  # noqa: E402
from paper_2005_08736_gb300.solver import Simulation, taylor_green_config  # noqa: E402

FP64_TOL = 1e-12


def rel_linf(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def noalloc_step(lib, cfg, state: "torch.Tensor", nsteps: int, dt: float = 0.0) -> None:
    c = cfg.c_struct()
    stream = torch.cuda.current_stream()
    status = lib.hgks_step_noalloc(ctypes.byref(c), ctypes.c_void_p(state.data_ptr()), nsteps,
                                   float(dt), ctypes.c_void_p(stream.cuda_stream))
    assert status == _lib.HGKS_OK, _lib.STATUS_NAMES.get(status, status)
    torch.cuda.synchronize()


@pytest.mark.parametrize("recon,flux", [("weno-z", "full"), ("linear", "smooth")])
def test_noalloc_step_matches_the_allocating_step_on_two_calls(recon, flux):
    lib = _lib.load()
    n = 20
    cfg = taylor_green_config(n, "fp64", recon, flux)
    Q0 = oracle.conservative(inputs.taylor_green(n), 1.4)
    dev = torch.from_numpy(np.ascontiguousarray(Q0)).to("cuda")
    sim = Simulation(cfg)
    sim.init_conservative(Q0)
    for _ in range(2):
        noalloc_step(lib, cfg, dev, 2)
        sim.step(2)
        err = rel_linf(dev.cpu().numpy(), sim.state())
        assert err <= FP64_TOL, err
    sim.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    lib = _lib.load()
    cfg = taylor_green_config(33, "fp64")
    dev = torch.zeros(cfg.shape, dtype=torch.float64, device="cuda")
    c = cfg.c_struct()
    status = lib.hgks_step_noalloc(ctypes.byref(c), ctypes.c_void_p(dev.data_ptr()), 1, 0.0, None)
    assert status == _lib.HGKS_E_UNSUPPORTED


def test_noalloc_rejects_the_mass_flux_force():
    # the force's FP64 partial sums need a buffer the static scratch does not hold
    lib = _lib.load()
    cfg = taylor_green_config(16, "fp64")
    cfg.force_mode, cfg.mass_flux = 1, 0.0
    dev = torch.zeros(cfg.shape, dtype=torch.float64, device="cuda")
    c = cfg.c_struct()
    status = lib.hgks_step_noalloc(ctypes.byref(c), ctypes.c_void_p(dev.data_ptr()), 1, 0.0, None)
    assert status == _lib.HGKS_E_UNSUPPORTED
