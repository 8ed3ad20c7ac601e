"""Host check of the integer TF32 rounding that the last contraction's split
uses (csrc/tf32_round.h), over all 2^32 FP32 bit patterns, against the
rounding's definition (round to nearest, ties away from zero, to 10 stored
mantissa bits; tests/tf32_round_check.cpp), and of the split x = hi + lo
with lo = x - hi exact in FP32.  The same header is compiled into the
kernels, so this pins the rounding the tensor-core path relies on without a
GPU."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_01180_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "tf32_round_check.cpp")


def test_tf32_rounding_and_split_exhaustive(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "tf32_round_check")
    # no -ffast-math: IEEE single-precision subtraction with subnormals, as on the GPU
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC, SRC, "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=600).stdout
    vals = {k: int(v) for k, v in re.findall(r"^(\w+) (\d+)", out, flags=re.M)}
    # every finite pattern rounds as the definition says
    assert vals["finite_mismatch"] == 0, out
    # hi + lo == x exactly whenever hi is finite (Sterbenz: x and hi within a factor 2)
    assert vals["split_inexact"] == 0, out
    # infinities and NaNs give a NaN lo, so they reach the sum as NaN
    assert vals["nonfinite_lo_finite"] == 0, out
    # only |x| >= (2 - 2^-11) 2^127 rounds past the largest TF32 value:
    # 2^12 mantissa patterns of the top binade, both signs
    assert vals["overflow_to_inf"] == 2 * 4096, out
