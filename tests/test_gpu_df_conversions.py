"""The library's integer conversions between float64 and double-float
(df64.cuh) give the float64 conversions' values bit for bit: a small CUDA
program (tests/cuda/df_conversion_check.cu) compiled against the library's
header checks 1.3e8 seeded values on the GPU."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2211_08948_gb300", "csrc")


def _nvcc():
    for c in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")]:
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not found")


def test_integer_conversions_equal_float64_conversions(tmp_path):
    exe = str(tmp_path / "df_conversion_check")
    src = os.path.join(HERE, "cuda", "df_conversion_check.cu")
    r = subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I" + CSRC,
                        src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "mismatches 0 " in r.stdout, r.stdout + r.stderr
