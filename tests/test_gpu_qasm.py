"""GPU parity of OpenQASM 2.0 imports (Sec. 3.3 "OpenQASM Integration";
App. B.1): programs parsed by qs_qasm_parse run through qs_apply_circuit in
both modes and match the complex128 oracle run on the same parsed records.

Programs (synthetic, written here): a layered circuit over two registers
with nested user-defined gates, register-wide calls, barriers and trailing
measurements; a cat state; a QFT written with cu1 and swaps; a QFT with
cu1 spelled out as u1 / cx.  Circuits of random CX . diagonal . CX blocks
check the detector's fold of such blocks.  Tolerances as
in the other parity tests: max |d| <= 2e-5, relative L2 <= 1e-5,
fidelity >= 1 - 1e-6."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_19147_gb300 as qs  # noqa: E402


def _layered(na, nb, layers, seed):
    rng = np.random.default_rng(seed)
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg a[{na}];", f"qreg b[{nb}];",
             f"creg c[{na + nb}];",
             "gate zz(t) x, y { cx x, y; rz(t) y; cx x, y; }",
             "gate layer(t, f) x, y { ry(f) x; rx(-f/2) y; zz(t*pi) x, y; }",
             "gate tof x, y, z { h z; cx y, z; tdg z; cx x, z; t z; cx y, z; tdg z; cx x, z; t y; t z; h z;"
             " cx x, y; t x; tdg y; cx x, y; }"]
    n = na + nb
    for _ in range(layers):
        lines.append("h a;")
        lines.append(f"layer({rng.uniform(-1, 1)!r}, {rng.uniform(-3, 3)!r}) a, b[{int(rng.integers(nb))}];")
        lines.append(f"cu1({rng.uniform(0, 2 * np.pi)!r}) a[{int(rng.integers(na))}], b[{int(rng.integers(nb))}];")
        u, v, w = (int(x) for x in rng.choice(n, size=3, replace=False))
        reg = lambda q: f"a[{q}]" if q < na else f"b[{q - na}]"
        lines.append(f"tof {reg(u)}, {reg(v)}, {reg(w)};")
        lines.append(f"u3({rng.uniform(0, 3)!r}, {rng.uniform(0, 3)!r}, {rng.uniform(0, 3)!r}) b;")
        lines.append("barrier a, b;")
    lines.append("measure a[0] -> c[0];")
    return "\n".join(lines) + "\n"


def _cat(n):
    return (f"OPENQASM 2.0;\nqreg q[{n}];\nh q[0];\n" + "".join(f"cx q[{i}], q[{i + 1}];\n" for i in range(n - 1)))


def _qft(n):
    s = f"OPENQASM 2.0;\ninclude \"qelib1.inc\";\nqreg q[{n}];\n"
    for j in range(n):
        s += f"h q[{j}];\n"
        for k in range(j + 1, n):
            s += f"cu1(pi/2^{k - j}) q[{k}], q[{j}];\n"
    for j in range(n // 2):
        s += f"swap q[{j}], q[{n - 1 - j}];\n"
    return s


def _decomposed_qft(n):
    # cu1 spelled out as u1 / cx (App. B.1), folded back into CPHASE by the detector
    s = f"OPENQASM 2.0;\ninclude \"qelib1.inc\";\nqreg q[{n}];\n"
    for g in W.spell_out_2q(W.qft_gates(n)):
        name = {"H": "h", "P": "u1", "CX": "cx", "SWAP": "swap"}[g.kind]
        prm = f"({g.params[0]!r})" if g.params else ""
        s += f"{name}{prm} " + ", ".join(f"q[{w}]" for w in g.wires) + ";\n"
    return s


@pytest.mark.parametrize("name,src,mode", [
    ("layered 10+8", _layered(10, 8, 6, 31), "fused"),
    ("layered 10+8", _layered(10, 8, 6, 31), "pergate"),
    ("layered 12+9", _layered(12, 9, 4, 32), "fused"),
    ("cat 22", _cat(22), "fused"),
    ("qft 19", _qft(19), "fused"),
    ("decomposed qft 18", _decomposed_qft(18), "fused"),
])
def test_imported_programs_match_oracle(name, src, mode):
    n, gates = qs.parse_qasm(src)
    psi0 = W.random_state(n, 7)
    st = qs.State(n)
    st.set(psi0.astype(np.complex64))
    st.apply(gates, mode=mode)
    got = st.get()[0].astype(np.complex128)
    st.close()
    ref = oracle.simulate(n, gates, psi0.astype(np.complex64).astype(np.complex128))
    d = np.max(np.abs(got - ref))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    assert d <= 2e-5 and rel <= 1e-5 and fid >= 1 - 1e-6, (name, d, rel, fid)


@pytest.mark.parametrize("n,seed", [(12, 1), (17, 2), (20, 3)])
def test_cx_sandwich_circuits_match_oracle(n, seed):
    # CX . diagonal . CX blocks folded into two-qubit diagonals by the detector
    gates = W.cx_sandwich_circuit(n, 80, 900 + seed)
    psi0 = W.random_state(n, seed)
    st = qs.State(n)
    st.set(psi0.astype(np.complex64))
    st.apply(gates)
    got = st.get()[0].astype(np.complex128)
    st.close()
    ref = oracle.simulate(n, gates, psi0.astype(np.complex64).astype(np.complex128))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert np.max(np.abs(got - ref)) <= 2e-5 and rel <= 1e-5, rel
