"""The split-precision GEMM's work order (csrc/oz_order.cuh, the header the
kernel includes), compiled on the host with g++: for full and lower outputs,
many tile grids and band widths, with one CTA per tile and with clusters of
two on tile-row pairs, every output tile is computed exactly once and the
launch's item count matches the order."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2605_21149_gb300", "csrc", "oz_order.cuh")


def test_split_gemm_work_order(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "oz_order_check"
    subprocess.run([cxx, "-O2", "-std=c++17", f'-DOZ_ORDER_HEADER="{HEADER}"',
                    os.path.join(HERE, "host", "oz_order_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout
