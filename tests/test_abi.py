"""The C ABI library loads and exports every entry point include/*.h declares;
struct layouts agree between C and the ctypes binding; configuration errors
are rejected on the host (CPU only: no kernel runs here)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2005_08736_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            src = open(os.path.join(INCLUDE, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(hgks_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert "hgks_step" in names and "hgks_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(hgks_\w+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    assert sorted(_lib.EXPORTS) == sorted(n for n in names if n in _lib.EXPORTS)


def test_struct_layouts_match_the_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "hgks.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(hgks_config), offsetof(hgks_config, prec),
         offsetof(hgks_config, p_ref), sizeof(hgks_diag), offsetof(hgks_diag, step),
         sizeof(hgks_turbulence), sizeof(hgks_channel), offsetof(hgks_channel, C_f));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", INCLUDE, c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    assert vals == [ctypes.sizeof(_lib.HgksConfig), _lib.HgksConfig.prec.offset,
                    _lib.HgksConfig.p_ref.offset, ctypes.sizeof(_lib.HgksDiag),
                    _lib.HgksDiag.step.offset, ctypes.sizeof(_lib.HgksTurbulence),
                    ctypes.sizeof(_lib.HgksChannel), _lib.HgksChannel.C_f.offset]


@pytest.mark.parametrize("field,value", [("nx", 5), ("nz", 65530), ("gamma", 1.0), ("prandtl", 0.0), ("cfl", -1.0),
                                         ("recon", 7), ("flux", 2), ("prec", 3), ("p_ref", 0.0),
                                         ("bc_y", 4), ("y_stretch", 1)])
def test_invalid_configurations_are_rejected_before_any_device_work(lib, field, value):
    reject(lib, {field: value})


def test_the_tanh_mapping_needs_the_channel_height_two(lib):
    reject(lib, {"bc_y": 1, "y_stretch": 1, "ly": 3.0, "y0": -1.5})


def reject(lib, fields):
    cfg = _lib.HgksConfig()
    assert lib.hgks_default_config(ctypes.byref(cfg), 16) == _lib.HGKS_OK
    for field, value in fields.items():
        setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.hgks_create(ctypes.byref(cfg), None, ctypes.byref(h)) == _lib.HGKS_E_INVAL
    assert not h.value
    assert lib.hgks_last_error(None)


def test_default_config_is_the_taylor_green_setting(lib):
    cfg = _lib.HgksConfig()
    assert lib.hgks_default_config(ctypes.byref(cfg), 32) == _lib.HGKS_OK
    assert (cfg.nx, cfg.gamma, cfg.prandtl, cfg.cfl) == (32, 1.4, 0.72, 0.5)
    assert cfg.mu_ref == pytest.approx(1 / 1600)
    assert cfg.p_ref == pytest.approx(100 / 1.4)
    assert lib.hgks_default_config(ctypes.byref(cfg), 5) == _lib.HGKS_E_INVAL


def test_null_arguments_are_rejected_before_any_device_work(lib):
    # The error behaviour the header states: a null context or output is
    # E_INVAL (destroying nothing is OK); no call reaches the device.
    E = _lib.HGKS_E_INVAL
    d = ctypes.c_double()
    i = ctypes.c_int()
    buf = (ctypes.c_double * 8)()
    cfg = _lib.HgksConfig()
    assert lib.hgks_default_config(ctypes.byref(cfg), 16) == _lib.HGKS_OK
    calls = [
        lib.hgks_default_config(None, 16),
        lib.hgks_create(ctypes.byref(cfg), None, None),
        lib.hgks_init_state(None, buf, 1),
        lib.hgks_init_conservative(None, buf, 1),
        lib.hgks_get_state(None, buf, 1),
        lib.hgks_step(None, 1, 0.0, 1, ctypes.byref(d)),
        lib.hgks_set_time(None, 0.0, 0),
        lib.hgks_diagnostics(None, ctypes.byref(_lib.HgksDiag())),
        lib.hgks_turbulence_stats(None, ctypes.byref(_lib.HgksTurbulence())),
        lib.hgks_channel_stats(None, buf, ctypes.byref(_lib.HgksChannel())),
        lib.hgks_adjoint_step(None, 0.1, buf, buf),
        lib.hgks_autotune(None, ctypes.byref(i), ctypes.byref(i), ctypes.byref(d)),
        lib.hgks_set_sweep_shape(None, 0, 0),
        lib.hgks_profile_step(None, 0.0, buf, 8),
        lib.hgks_ensemble_create(None, 1, None),
        lib.hgks_ensemble_step(None, 1, 0.0, 1),
        lib.hgks_step_noalloc(None, buf, 1, 0.0, None),
        lib.hgks_step_noalloc(ctypes.byref(cfg), None, 1, 0.0, None),
        lib.hgks_step_noalloc(ctypes.byref(cfg), buf, -1, 0.0, None),
        lib.hgks_measure_fp_peaks(None, None),
    ]
    assert calls == [E] * len(calls)
    assert lib.hgks_destroy(None) == _lib.HGKS_OK
    assert lib.hgks_ensemble_destroy(None) == _lib.HGKS_OK
    assert lib.hgks_last_error(None)
    assert lib.hgks_ensemble_last_error(None) == b""


def test_allocation_free_step_limits_are_checked_on_the_host(lib):
    # hgks_step_noalloc: an invalid configuration is E_INVAL, a grid above its
    # fixed capacity or the constant-mass-flux force is E_UNSUPPORTED, all
    # before any device call.
    buf = (ctypes.c_double * 8)()
    for fields, status in (({"gamma": 1.0}, _lib.HGKS_E_INVAL),
                           ({"nx": 33}, _lib.HGKS_E_UNSUPPORTED),
                           ({"force_mode": 1}, _lib.HGKS_E_UNSUPPORTED)):
        cfg = _lib.HgksConfig()
        assert lib.hgks_default_config(ctypes.byref(cfg), 16) == _lib.HGKS_OK
        for k, v in fields.items():
            setattr(cfg, k, v)
        assert lib.hgks_step_noalloc(ctypes.byref(cfg), buf, 1, 0.0, None) == status
