"""The projection kernels' exact-arithmetic helpers (csrc/exact.cuh), built
for the host with g++ and checked against plain FP64 arithmetic by
tests/exact_helpers_check.cpp: the order-free sums' quantisation of an FP32
value without FP64 arithmetic, the integer FP64 -> FP32 rounding and
finiteness test of the per-pair round control, and the exact FP32 TwoSum
maximum of |X(t+1) - X(t)| behind the outer stop (Algorithm 1).  The kernels
compile the same source for the device (bit views by intrinsics instead of
memcpy)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1207_1114_gb300", "csrc")


def test_exact_helpers_match_fp64_arithmetic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "exact_helpers_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "exact_helpers_check.cpp"),
                    "-o", exe], check=True, capture_output=True, text=True)
    r = subprocess.run([exe, "1000000"], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("mismatches 0 of") == 3
