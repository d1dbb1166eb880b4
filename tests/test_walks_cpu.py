"""Host check of the FP32 kernel's walker programs (csrc/walks.cpp): tests/walks_check.cpp
replays every walker's steps on column sets for the operator library's e-graph plans (both
flavours, several walker counts and batch sizes) and checks the leaf column sets, Laplace
signs, single coverage of every leaf, batch sizes and cost balance (CPU, g++)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2201_04269_gb300", "csrc")


def test_walker_programs(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    exe = str(tmp_path / "walks_check")
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CSRC}", os.path.join(ROOT, "tests", "walks_check.cpp"),
                    os.path.join(CSRC, "walks.cpp"), os.path.join(CSRC, "planner.cpp"), "-o", exe],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
