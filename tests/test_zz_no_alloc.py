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
from paper_2005_08736_gb300.solver import Config, Simulation, taylor_green_config  # noqa: E402

FP64_TOL = 1e-12
# The FP32 tolerance of the parity tests (per variable; the momentum
# components share the largest momentum magnitude as their scale).
FP32_TOL = 2e-5


def rel_linf(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def rel_linf_shared(a, b):
    scale = [max(np.abs(b[v]).max(), 1e-300) for v in range(5)]
    scale[1:4] = [max(scale[1:4])] * 3
    return max(np.abs(a[v] - b[v]).max() / scale[v] for v in range(5))


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


def compare_two_calls(cfg, prim, nsteps=2, tol=FP64_TOL):
    """Two noalloc calls in a row against the allocating context stepped alike."""
    lib = _lib.load()
    Q0 = oracle.conservative(prim, cfg.gamma)
    dev = torch.from_numpy(np.ascontiguousarray(Q0)).to("cuda")
    sim = Simulation(cfg)
    sim.init_conservative(Q0)
    errs = []
    for _ in range(2):
        noalloc_step(lib, cfg, dev, nsteps)
        sim.step(nsteps)
        ref = sim.state()
        errs.append(rel_linf(dev.cpu().numpy(), ref) if tol == FP64_TOL
                    else rel_linf_shared(dev.cpu().numpy(), ref))
    sim.close()
    assert max(errs) <= tol, errs


def test_noalloc_fp32_matches_the_allocating_fp32_step():
    # FP32: the per-call clearing of the compensation buffer and the x sweep
    # reading the state directly (the allocating context reads a transposed copy)
    compare_two_calls(taylor_green_config(20, "fp32"), inputs.taylor_green(20), tol=FP32_TOL)


def test_noalloc_odd_grid_matches_the_allocating_step():
    # odd padded x extent: the x sweep's per-layer loads instead of pair loads
    n = (15, 17, 13)
    cfg = Config(*n, prec=0, recon=2, flux=1, tau_num_C=1.0, mu_ref=2e-3, p_ref=1.0)
    compare_two_calls(cfg, inputs.random_smooth(n, seed=61, amp=0.2))


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_noalloc_characteristic_variables_match_the_allocating_step(prec, tol):
    n = (14, 12, 10)
    cfg = Config(*n, prec=prec, recon=1, flux=1, tau_num_C=1.0, mu_ref=2e-3, p_ref=1.0,
                 recon_vars=1)
    compare_two_calls(cfg, inputs.random_smooth(n, seed=62, amp=0.2), tol=tol)


def test_noalloc_stretched_channel_matches_the_allocating_step():
    # the cell widths of the tanh mapping and the mirrored wall ghosts are
    # formed on the device by this entry point, separately from hgks_create
    n = (16, 20, 12)
    cfg = Config(*n, lx=2 * np.pi, ly=2.0, y0=-1.0, lz=np.pi, y_stretch=1, stretch_b=2.0, bc_y=1,
                 T_wall=100 / 1.4, mu_ref=0.0541 / 180, force_x=2.93e-3, prec=0)
    compare_two_calls(cfg, inputs.channel(*n, seed=4))


def test_noalloc_call_leaves_device_free_memory_unchanged():
    lib = _lib.load()
    cfg = taylor_green_config(24, "fp32", "weno-z", "full")
    Q0 = oracle.conservative(inputs.taylor_green(24), 1.4)
    dev = torch.from_numpy(np.ascontiguousarray(Q0)).to("cuda")
    noalloc_step(lib, cfg, dev, 1)  # loads the kernels this configuration uses
    free0, _ = torch.cuda.mem_get_info()
    noalloc_step(lib, cfg, dev, 2)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
