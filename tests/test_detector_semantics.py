"""The fusion detector's ops (and the dense-block regrouping) reproduce the
gate-by-gate product, checked on the host in complex128: a C++ program links
the planner, applies the detector's ops by their definitions and compares
with applying every gate's full matrix in order.  Circuits: random gate lists
over the whole vocabulary (n = 1..9), QFTs, Trotter and Heisenberg layers,
QAOA layers, CNOT ladders and GHZ chains, and circuits whose two-qubit
diagonals are spelled out as CX . diagonal . CX (folded by the detector)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from gate_text import gate_lines

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__._build_lib_module().build()
    import paper_2609_19147_gb300 as m
    return m


def _circuits():
    out = []
    rng = np.random.default_rng(17)
    for n in range(1, 10):
        for s in range(4):
            out.append((n, W.random_circuit(n, 30 + 10 * s, 1000 * n + s)))
    for n in (3, 6, 9):
        out.append((n, W.qft_gates(n, swaps=True)))
        out.append((n, W.tfim_gates(n, 3, 0.1, 1.0, W.tfim_fields(n, 3), order=2)))
        out.append((n, W.tfim_gates(n, 2, 0.1, 1.0, 0.7, order=1)))
        out.append((n, W.cnot_ladder(n) + W.ghz_gates(n)))
        hz = []
        for b in range(n - 1):
            t = float(rng.uniform(0, 1))
            hz += [W.Gate("RXX", (b, b + 1), (t,)), W.Gate("RYY", (b, b + 1), (t,)), W.Gate("RZZ", (b, b + 1), (t,))]
        out.append((n, hz))
    for n in (4, 6, 8):
        edges = W.random_regular3_graph(n, rng)
        out.append((n, W.qaoa_gates(n, edges, [0.4, 1.1], [0.7, 0.2])))
        out.append((n, W.spell_out_2q(W.qaoa_gates(n, edges, [0.4], [0.7]))))
    # decomposed two-qubit diagonals (CX . diagonal . CX), folded by the detector
    for n in (3, 6, 9):
        out.append((n, W.spell_out_2q(W.qft_gates(n, swaps=True))))
        out.append((n, W.spell_out_2q(W.tfim_gates(n, 2, 0.1, 1.0, 0.7, order=2))))
    for n in range(2, 10):
        out.append((n, W.cx_sandwich_circuit(n, 40, 500 + n)))
    return out


def test_detector_ops_match_gate_product(tmp_path, qs):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir("/usr/local/cuda/include"):
        pytest.skip("needs g++ and the CUDA headers")
    lines = []
    for n, gl in _circuits():
        gl_text = gate_lines(qs, gl)
        lines.append(f"n {n} {len(gl_text)}")
        lines += gl_text
    src = tmp_path / "circuits.txt"
    src.write_text("\n".join(lines) + "\n")
    csrc = os.path.join(ROOT, "paper_2609_19147_gb300", "csrc")
    exe = str(tmp_path / "check")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                           "-I", "/usr/local/cuda/include",
                           os.path.join(ROOT, "tests", "cpp", "detector_semantics_check.cpp"),
                           os.path.join(csrc, "qs_plan.cpp"), "-o", exe, "-lpthread"])
    out = subprocess.run([exe, str(src)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
    f = out.stdout.split()
    assert int(f[1]) == len(_circuits())
    counts = [int(x) for x in f[3:9]]      # U1, U2, DIAG, QFT, GF2, DENSE: every op kind was exercised
    assert all(c > 0 for c in counts), out.stdout
