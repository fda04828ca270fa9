"""The reverse-mode value cotangents of the full flux's parts (csrc/flux_rev.cuh,
used by the adjoint step) against forward-mode dual numbers through the
forward functions, on 200 seeded states, both half spaces and the
equilibrium part, constant and power-law viscosity, in double precision on
the host (the device formulas compile for the host too).  No GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reverse_value_cotangents_match_forward_mode(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "flux_vjp_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2005_08736_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-x", "cu",
                    os.path.join(ROOT, "tests", "support", "flux_vjp_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    worst = float(subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip())
    assert worst < 1e-12, worst
