"""The double-float arithmetic of the serendipity kernels (FP32 pairs for the
geometry, the Gram sums and the conversion back to FP64), compiled for the
host from the kernels' own header and checked against FP64: reciprocal and
square root by one Newton step within 2^-45, the integer FP32 -> FP64
conversion exact (zeros, infinities, the FP32 range), and the 27-point
geometry of jittered bricks at three scales within 1e-13 of FP64."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def check_output(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("dfc") / "df_arith_check")
    src = os.path.join(ROOT, "tests", "native", "df_arith_check.cu")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2111_03541_gb300", "csrc"), "-o", exe, src],
                   check=True, capture_output=True)
    return subprocess.run([exe], check=True, capture_output=True, text=True).stdout


def _num(out, key):
    return float(re.search(key + r"\s+([0-9.eE+-]+)", out).group(1))


def test_geometry_within_1e13(check_output):
    assert _num(check_output, "w detJ") < 1e-13
    assert _num(check_output, r"scaled\)") < 1e-13


def test_reciprocal_sqrt_and_conversion(check_output):
    assert _num(check_output, "recip max rel err") < 2.0 ** -45
    assert _num(check_output, r"sqrt") < 2.0 ** -45
    assert _num(check_output, "exact conversion mismatches") == 0
