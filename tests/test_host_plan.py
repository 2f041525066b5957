"""Launch-planning arithmetic (csrc/ld_plan.h) on the host: the C++ check
program tests/host/plan_check.cpp, built with the host compiler (no GPU, no
CUDA), pins D (Sec. 2.3) to the workloads' values, the Q16 table (Sec. 3.3)
to its end points and the unit circle, the interleaved accumulator's row
count to a brute force over every pixel, and the tile balancing and piece
splits to hand-worked cases (including an empty plan list)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_plan_arithmetic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "plan_check")
    src = os.path.join(HERE, "host", "plan_check.cpp")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-o", exe, src], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all passed" in r.stdout
