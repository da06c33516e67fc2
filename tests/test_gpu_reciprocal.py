"""The integration takes its quotients u = fx X / Z and v = fy Y / Z from one
reciprocal of Z per voxel, computed from the hardware's approximate
reciprocal and one Newton-Raphson step.  The quotients are exact only if that
reciprocal is the correctly rounded one; this test checks it against the IEEE
reciprocal on every float of the range the kernels use it on (the kernels
take IEEE divisions for any other Z)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.gpu
def test_newton_reciprocal_is_the_ieee_reciprocal(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "rcp_check")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-fmad=false",
                           "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_1708_00783_gb300", "csrc"),
                           os.path.join(HERE, "rcp_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300, check=True).stdout.split()
    assert out == ["0", "0"], out
