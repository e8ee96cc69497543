"""The planner's count-table diagonals (MK_DIAGC) checked on the host: a
small C++ program links the planner, builds plans for uniform RZZ / CP edge
sets with a uniform single-qubit RZ, and evaluates every emitted op's table
index for random amplitudes against the phase from the gate definitions."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_count_table_ops_match_gate_phases(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    cuda_inc = next((p for p in ("/usr/local/cuda/include",) if os.path.isdir(p)), None)
    if cuda_inc is None:
        pytest.skip("needs the CUDA headers")
    csrc = os.path.join(ROOT, "paper_2609_19147_gb300", "csrc")
    exe = str(tmp_path / "check")
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                           "-I", cuda_inc, os.path.join(ROOT, "tests", "cpp", "plan_count_table_check.cpp"),
                           os.path.join(csrc, "qs_plan.cpp"), "-o", exe, "-lpthread"])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
