"""Decomposed two-qubit diagonals (App. B.1: an imported QFT arrives as
cx + rz / u1 sequences and no longer fuses).  The detector folds every
CX(c,t) . [diagonals on c, t; gates elsewhere] . CX(c,t) sandwich, with the
diagonal runs next to it, into one two-qubit diagonal, so circuits written
that way plan exactly like the native ones: the same passes, micro-ops and
constants (the fold reproduces CPHASE and RZZ exactly).  The folded plans'
results are checked against the oracle on the host in
test_detector_semantics.py and test_plan_interpret.py, and on the GPU in
test_gpu_qasm.py."""
import pytest

import workloads as W


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__._build_lib_module().build()
    import paper_2609_19147_gb300 as m
    return m


def _body(txt):
    return txt.split("\n", 1)[1]   # without the header line (which counts the input gates)


@pytest.mark.parametrize("n", [12, 18, 24, 30])
def test_spelled_out_qft_plans_as_native(qs, n):
    nat, spelled = W.qft_gates(n), W.spell_out_2q(W.qft_gates(n))
    assert len(spelled) == len(nat) + 4 * (n * (n - 1) // 2)
    (tn, pn), (ts, ps) = qs.plan_describe(n, nat), qs.plan_describe(n, spelled)
    assert ps == pn and _body(ts) == _body(tn)
    assert "QFT=" in ts and ts.count("TILE") == pn - 1   # the stages fuse; the swaps are one permutation


@pytest.mark.parametrize("family", ["tfim", "qaoa", "heisenberg"])
def test_spelled_out_layers_plan_as_native(qs, family):
    import numpy as np
    n = 22
    if family == "tfim":
        nat = W.tfim_gates(n, 20, 0.05, 1.0, W.tfim_fields(n, 3), order=2)
    elif family == "qaoa":
        nat = W.qaoa_gates(n, W.random_regular3_graph(n, np.random.default_rng(4)), [0.3, 0.9], [0.5, 0.2])
    else:
        nat = []
        for b in range(n - 1):
            nat += [W.Gate("RXX", (b, b + 1), (0.1,)), W.Gate("RYY", (b, b + 1), (0.1,))]
        nat += [W.Gate("RZZ", (b, b + 1), (0.1,)) for b in range(n - 1)]
    spelled = W.spell_out_2q(nat)
    assert len(spelled) > len(nat)
    for kw in ({}, {"tile_qubits": 12, "group_qubits": 4}, {"tile_qubits": 13, "group_qubits": 5}):
        (tn, pn), (ts, ps) = qs.plan_describe(n, nat, **kw), qs.plan_describe(n, spelled, **kw)
        assert ps == pn and _body(ts) == _body(tn), (family, kw)


def test_imported_decomposed_qft_fuses(qs):
    # App. B.1's non-win: a QFT imported with cu1 spelled out as u1 / cx; now planned as the native QFT
    n = 18
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg q[{n}];"]
    for g in W.spell_out_2q(W.qft_gates(n)):
        name = {"H": "h", "P": "u1", "CX": "cx", "SWAP": "swap"}[g.kind]
        prm = f"({g.params[0]!r})" if g.params else ""
        lines.append(f"{name}{prm} " + ", ".join(f"q[{w}]" for w in g.wires) + ";")
    nq, parsed = qs.parse_qasm("\n".join(lines) + "\n")
    assert nq == n
    (tn, pn), (ti, pi) = qs.plan_describe(n, W.qft_gates(n)), qs.plan_describe(n, parsed)
    assert pi == pn and _body(ti) == _body(tn)


def test_sandwich_circuits_need_fewer_passes(qs):
    # random sandwiches: the fold turns CX pairs (gathers or controlled ops) into diagonals
    for n in (8, 16):
        gl = W.cx_sandwich_circuit(n, 60, 700 + n)
        _, p = qs.plan_describe(n, gl)
        assert p <= 12, p
