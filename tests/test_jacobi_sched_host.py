"""The float32 Jacobi phase's index arithmetic (csrc/jacobi_sched.cuh, the
header the kernel includes), compiled on the host with g++: pair ownership,
the columns' moves between rounds against the round-robin schedule, and the
next round's rotation inputs (each written exactly once, from the right
entry)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2605_21149_gb300", "csrc", "jacobi_sched.cuh")


def test_jacobi_schedule_index_arithmetic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "jacobi_sched_check"
    subprocess.run([cxx, "-O2", "-std=c++17", f'-DJACOBI_SCHED_HEADER="{HEADER}"',
                    os.path.join(HERE, "host", "jacobi_sched_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout
