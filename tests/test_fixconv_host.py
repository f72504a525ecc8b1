"""The split product's int64 -> float64 conversion (csrc/fixconv.cuh),
compiled on the host with g++ and compared bit for bit with the C++
(double) cast and ldexp: round to nearest with ties to even, signs, the
INT64_MIN edge, exponent overflow and underflow reported for the caller's
fallback."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2605_21149_gb300", "csrc", "fixconv.cuh")


def test_fixconv_matches_cast(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "fixconv_check"
    subprocess.run([cxx, "-O2", "-std=c++17", f'-DFIXCONV_HEADER="{HEADER}"',
                    os.path.join(HERE, "host", "fixconv_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout
