"""Double-float (df64) arithmetic used by the optional inner-region path: compiled for the
host with nvcc and checked against long double on seeded random operands (sin and cos both
by argument reduction and by the node table the geodesic steps use, over [0, 1.02 pi] so
that the fallback is exercised too).  CPU only."""
import json
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "df64_check.cu")
INC = os.path.join(ROOT, "paper_1801_10452_b300", "csrc")


def test_df64_accuracy(tmp_path):
    exe = str(tmp_path / "df64_check")
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", INC, "-o", exe, SRC], check=True, capture_output=True)
    r = json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)
    # a 48-bit significand: a few units of 2^-48 = 3.6e-15 per operation
    for k in ("add", "mul", "div", "sqrt", "sin_abs", "cos_abs", "sincos_table_abs"):
        assert r[k] < 3e-14, (k, r[k])
