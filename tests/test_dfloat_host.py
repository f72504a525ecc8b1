"""Float-float helpers of the split Cholesky's opt-in diagonal blocks
(csrc/dfloat.cuh), checked on the host: the header's own function bodies are
compiled with g++ (CUDA intrinsics mapped to IEEE float32 round-to-nearest
operations, fma contraction off) against long-double arithmetic.  Bounds:
conversion 2^-47, product and multiply-subtract 2^-45 (relative to the
operands' magnitudes for the latter), reciprocal square root 2^-45 (Dekker's
product and Knuth's TwoSum are exact, so a few roundings of 2^-48 remain)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2605_21149_gb300", "csrc", "dfloat.cuh")


def test_dfloat_error_bounds(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    text = open(HEADER).read()
    body = text[text.index("namespace qmlgb {") + len("namespace qmlgb {"):
                text.rindex("}  // namespace qmlgb")]
    inc = tmp_path / "dfloat_body.inc"
    inc.write_text(body)
    exe = tmp_path / "dfloat_check"
    subprocess.run([cxx, "-O1", "-std=c++17", "-ffp-contract=off",
                    f'-DDFLOAT_BODY="{inc}"', os.path.join(HERE, "host", "dfloat_check.cpp"),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
