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

import numpy as np
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


def _tf32_rna(u):
    # the header's expression on uint32 arrays (its exhaustive check is above)
    return (u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)


def test_split_error_bound_and_no_coherent_bias():
    # The tensor core reads a TF32 operand's leading bits, i.e. it truncates
    # the unrounded lo = x - hi to TF32.  Under that model the represented
    # value hi + trunc(lo) is within 2^-23 |x| of x (lo has at most 12
    # significant bits, the MMA drops at most the last), and since lo's sign
    # follows the rounding direction of hi (not the sign of x) the error has
    # no coherent sign: its mean relative to x vanishes, where a split that
    # truncates hi itself shrinks x by about 0.3 x 2^-22 on average.
    rng = np.random.default_rng(0)
    n = 1 << 22
    # normal FP32 values of both signs over a wide exponent range, random mantissas
    x = (rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-60, 60, n))).astype(np.float32)
    x *= np.where(rng.random(n) < 0.5, -1.0, 1.0).astype(np.float32)
    u = x.view(np.uint32)
    hi = _tf32_rna(u).view(np.float32)
    lo = (x - hi).astype(np.float32)
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), x.astype(np.float64))
    lo_mma = (lo.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    rel = (x.astype(np.float64) - hi - lo_mma) / np.abs(x.astype(np.float64))
    assert np.abs(rel).max() <= 2.0 ** -23
    # signed error toward zero, relative to |x|: positive = shrink
    shrink = rel * np.sign(x.astype(np.float64))
    # the truncating split for comparison: hi = trunc(x), lo = x - hi, lo truncated
    hi_t = (u & np.uint32(0xFFFFE000)).view(np.float32)
    lo_t = ((x - hi_t).astype(np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    shrink_t = (x.astype(np.float64) - hi_t - lo_t) / np.abs(x.astype(np.float64)) * np.sign(x)
    assert shrink_t.mean() > 0.25 * 2.0 ** -22                 # coherent shrink
    assert abs(shrink.mean()) < 0.01 * shrink_t.mean()         # none for this split
