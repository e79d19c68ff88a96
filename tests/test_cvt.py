"""The integer-pipe double -> float / float-float conversions (csrc/cvt.cuh) must round exactly
as IEEE 754 round-to-nearest-even does: checked on the host, bit for bit, over every exponent,
the rounding boundaries of the dropped significand bits (ties to even, carries into the
exponent), zeros, subnormals, infinities and nan (tests/cvt_check.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1602_02313_gb300", "csrc")


def test_integer_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "cvt_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "cvt_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    assert "0 mismatches" in r.stdout
