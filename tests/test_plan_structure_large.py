"""Plans for large states (26-33 qubits: the bench's 30-qubit launch
configuration, the 28-qubit suite, the 25-qubit sweep, the 33-qubit maximum),
checked on the host without a state: every pass builds, every descriptor keeps
its invariants (sweep bits, table limits, constant bounds and alignment,
swizzled offsets), the tensor-copy box of 8 sampled tiles per pass (the first,
the last, six pseudo-random ones; with the batch coordinate for batched plans) covers
exactly that tile, inside the tensor, with 16-byte strides and an aligned
innermost coordinate, and the sweeps run on a zero tile of each."""
import numpy as np
import pytest

import plan_host
import workloads as W


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__._build_lib_module().build()
    import paper_2609_19147_gb300 as m
    return m


def _cases():
    out = []
    for n in (26, 30, 33):
        out.append((f"qft{n}", n, W.qft_gates(n), (0, 0, 0, 0, 0)))
        out.append((f"tfim{n}", n, W.tfim_gates(n, 3, 0.05, 1.0, W.tfim_fields(n, 3), order=2), (0, 0, 0, 0, 0)))
    for T, L, R in ((12, 4, 4), (13, 4, 5), (13, 5, 4), (12, 5, 5), (10, 3, 3)):
        out.append((f"tfim30 {T},{L},{R}", 30, W.tfim_gates(30, 3, 0.05, 1.0, W.tfim_fields(30, 3), order=2),
                    (T, L, R, 0, 0)))
    out.append(("qft30 12,4,4", 30, W.qft_gates(30), (12, 4, 4, 0, 0)))
    out.append(("suite28", 28, W.suite28_gates(28, 3, 1, tail=True), (0, 0, 0, 0, 0)))
    for prec in (1, 2, 3):
        out.append((f"dense{prec} tfim30", 30, W.tfim_gates(30, 2, 0.05, 1.0, W.tfim_fields(30, 3), order=2),
                    (13, 4, 5, prec, 5)))
    for name, gl in W.sweep_workloads(25):
        out.append((f"sweep {name}", 25, gl, (0, 0, 0, 0, 0)))
    vqe = W.vqe_ansatz_gates(24, 2)
    out.append(("vqe24 batch", 24, vqe, (0, 0, 0, 0, 0), W.vqe_params(24, 2, 3, 6)))
    out.append(("random33", 33, W.random_circuit(33, 200, 5), (0, 0, 0, 0, 0)))
    return out


def test_large_plans_keep_their_invariants(tmp_path, qs):
    if not plan_host.available():
        pytest.skip("needs g++ and the CUDA headers")
    cases = _cases()
    res = plan_host.interpret(qs, cases, str(tmp_path), [None] * len(cases))
    tma = sum(c["tma"] for _, c in res)
    rows = sum(c["rows"] for _, c in res)
    assert tma > 100 and rows >= 0
    merged = [c["merged"] for (name, *_), (_, c) in zip(cases, res) if name == "vqe24 batch"]
    assert merged == [1]
