"""hgks_count_flops: the algorithmic operation tally of one face of the sweep
kernel (host arithmetic only; no GPU needed).

The tally runs the kernel's closed forms on the host with a counting number
type.  Pins: the tangential pass with linear weights against a count written
out by hand from its formulas (recon.cuh: the quartic's values E -+ O and
derivatives A -+ B at the two Gauss abscissae), precision independence,
orderings that must hold between the modes, and the argument checks.
"""
import ctypes

import pytest

from paper_2005_08736_gb300 import _lib
from paper_2005_08736_gb300.solver import isotropic_config, taylor_green_config

NAMES = ["add", "mul", "div", "sqrt", "exp", "erf", "pow"]


@pytest.fixture(scope="module")
def lib():
    try:
        return _lib.load()
    except (RuntimeError, OSError) as e:  # library not built, or no CUDA runtime
        pytest.skip(str(e))


def tally(lib, cfg, stage=1):
    out = (ctypes.c_double * 21)()
    st = lib.hgks_count_flops(ctypes.byref(cfg.c_struct()), stage, out)
    assert st == _lib.HGKS_OK
    return [dict(zip(NAMES, out[7 * p:7 * p + 7])) for p in range(3)]


def flops(part):
    return part["add"] + part["mul"] + part["div"]


def test_linear_t1_pass_matches_the_hand_count(lib):
    # One field's quartic at both Gauss abscissae, values and derivatives:
    #   E = 719/720 f2 + (f1+f3)/1080 - (f0+f4)/4320        3 mul, 4 add
    #   O = sqrt3 (7/432 (f0-f4) + 25/216 (f3-f1))          3 mul, 3 add
    #   A = (f0-f4)/12 + 2/3 (f3-f1)  (differences shared)  2 mul, 1 add
    #   B = sqrt3/54 (-f0 + 13 f1 - 24 f2 + 13 f3 - f4)     4 mul, 4 add
    #   E -+ O, A -+ B                                            4 add
    # values only: E, O and E -+ O                           6 mul, 9 add.
    # The smooth flux's t1 pass: 5 state fields (values and derivatives)
    # and their 5 normal slopes (values only).
    t = tally(lib, taylor_green_config(32, "fp32"))[1]
    assert t["mul"] == 5 * 12 + 5 * 6
    assert t["add"] == 5 * 16 + 5 * 9
    assert t["div"] == t["sqrt"] == t["exp"] == t["erf"] == 0


def test_tally_is_independent_of_the_precision(lib):
    for recon, flux in (("linear", "smooth"), ("weno-z", "full")):
        a = tally(lib, taylor_green_config(32, "fp32", recon, flux))
        b = tally(lib, taylor_green_config(32, "fp64", recon, flux))
        assert a == b


def test_tally_orderings(lib):
    ls = [flops(p) for p in tally(lib, taylor_green_config(32, "fp32"))]
    ls2 = [flops(p) for p in tally(lib, taylor_green_config(32, "fp32"), stage=2)]
    wz = [flops(p) for p in tally(lib, taylor_green_config(32, "fp32", "weno-z", "smooth"))]
    full = [flops(p) for p in tally(lib, isotropic_config(32, "fp32"))]
    assert all(x > 0 for x in ls)
    # stage 2 stores dF only: same face fields and t1 pass, less flux work
    assert ls2[:2] == ls[:2] and ls2[2] < ls[2]
    # nonlinear weights cost more than the linear ones in every part
    assert all(w > l for w, l in zip(wz, ls))
    # the full flux needs three states at every Gauss point
    assert full[1] == 3 * wz[1] and full[2] > 3 * wz[2] / 2
    # the compatibility state needs erf and exp once per side of the face
    p0 = tally(lib, taylor_green_config(32, "fp32"))[0]
    assert p0["erf"] == 2 and p0["exp"] == 2


def test_count_arguments_are_checked(lib):
    out = (ctypes.c_double * 21)()
    c = taylor_green_config(32, "fp32").c_struct()
    assert lib.hgks_count_flops(ctypes.byref(c), 3, out) == _lib.HGKS_E_INVAL
    assert lib.hgks_count_flops(None, 1, out) == _lib.HGKS_E_INVAL
    ch = taylor_green_config(32, "fp32", "weno-z", "full", recon_vars=1).c_struct()
    assert lib.hgks_count_flops(ctypes.byref(ch), 1, out) == _lib.HGKS_E_UNSUPPORTED
