"""The integer-based binary64 <-> binary32 conversions the density kernel uses
for its FP64 records (csrc/tb_fpconv.cuh), compiled for the host and checked
against the C++ conversions on 2e6 random doubles across the binary32 range
(within half an ulp, ties at most one ulp away; f2d exact) and the special
values (signed zeros, overflow to infinity, flushed subnormals, NaN)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_0910_4497_gb300", "csrc")


def test_fp_conversions_match_the_hardware(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "fpconv_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "fpconv_check.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
