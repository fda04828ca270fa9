"""The packed FP32-pair reconstructions and transposes (csrc/packed.cuh,
csrc/adjoint.cuh: WENO5 end values, tangential values and derivatives with
linear, WENO-JS and WENO-Z weights, and the transposes of the nonlinear
ones) against the scalar functions they restate, half by half, on 2000
seeded FP32 stencils from near-linear to strongly nonlinear weights and
on constant stencils.  Built for the host (a pair operation is then the two
scalar operations), so this checks the packed algebra without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_packed_pairs_match_the_scalar_functions(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "packed_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                    "-I", os.path.join(ROOT, "paper_2005_08736_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-x", "cu",
                    os.path.join(ROOT, "tests", "support", "packed_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    fwd, rev = (float(x) for x in subprocess.run([exe], check=True, capture_output=True,
                                                 text=True).stdout.split())
    # FP32 rounding of the reconstructions; the transposes' amplified rounding
    # (the scalar FP32 transpose is ~3e-5 from FP64 on these stencils)
    assert fwd < 1e-5, fwd
    assert rev < 2e-4, rev
