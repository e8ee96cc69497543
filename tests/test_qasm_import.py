"""OpenQASM 2.0 import (Sec. 3.3 "OpenQASM Integration"; App. B.1) through
qs_qasm_parse, on the CPU.

* Programs written from the seeded workload generators parse back to the same
  gate records, and the oracle evolves both to the same state.
* User-defined gates (nested, with parameter expressions) inline to gates
  whose product the oracle checks against the gate they spell out (Toffoli
  from H / T / CX, CPHASE from U1 / CX, the Sec. 5.1 ZZ term from CX / RZ),
  equal up to the global phase their textual form carries.
* Register-wide calls broadcast; barriers are skipped; trailing measurements
  are accepted; every documented error comes back with its status and line.
* Imported circuits fuse as the native ones do (App. B.1): GHZ and cat-state
  CNOT chains become one gather, a QFT written with cu1 plans the same passes
  as the generator's QFT."""
import numpy as np
import pytest

import oracle
import workloads as W

QASM_NAME = {"I": "id", "X": "x", "Y": "y", "Z": "z", "H": "h", "S": "s", "SDG": "sdg", "T": "t", "TDG": "tdg",
             "SX": "sx", "RX": "rx", "RY": "ry", "RZ": "rz", "P": "u1", "U2": "u2", "U3": "u3", "CX": "cx",
             "CY": "cy", "CZ": "cz", "CH": "ch", "SWAP": "swap", "ISWAP": "iswap", "CRX": "crx", "CRY": "cry",
             "CRZ": "crz", "CP": "cu1", "RZZ": "rzz", "RXX": "rxx", "RYY": "ryy", "CCX": "ccx", "CSWAP": "cswap"}


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__._build_lib_module().build()
    import paper_2609_19147_gb300 as m
    return m


def to_qasm(n, gates, reg="q"):
    """A gate list as an OpenQASM 2.0 program on one register (angles as exact decimal)."""
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg {reg}[{n}];"]
    for g in gates:
        args = ", ".join(f"{reg}[{w}]" for w in g.wires)
        prm = "(" + ", ".join(repr(float(p)) for p in g.params) + ")" if g.params else ""
        lines.append(f"{QASM_NAME[g.kind]}{prm} {args};")
    return "\n".join(lines) + "\n"


def _state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    return v / np.linalg.norm(v)


def _same_up_to_phase(a, b, tol=1e-12):
    ov = np.vdot(a, b)
    return abs(abs(ov) - 1.0) < tol and np.allclose(a * ov / abs(ov), b, atol=tol)


def test_generated_programs_round_trip(qs):
    kinds = [k for k in QASM_NAME]
    cases = [(n, W.random_circuit(n, 120, 40 + n, kinds=kinds)) for n in (3, 5, 8)]
    cases += [(10, W.qft_gates(10)), (9, W.tfim_gates(9, 3, 0.1, 1.0, W.tfim_fields(9, 3), order=2)),
              (8, W.suite28_gates(8, 2, 3, tail=False))]
    for n, gl in cases:
        gl = [g for g in gl if g.kind != "U"]   # a dense 2x2 has no OpenQASM name
        nq, parsed = qs.parse_qasm(to_qasm(n, gl))
        assert nq == n and len(parsed) == len(gl)
        for a, b in zip(parsed, gl):
            assert a.kind == b.kind and tuple(a.wires) == tuple(b.wires)
            assert np.array_equal(np.asarray(a.params, float), np.asarray(b.params, float))
        psi0 = _state(n, n)
        assert np.array_equal(oracle.simulate(n, parsed, psi0), oracle.simulate(n, gl, psi0))


def test_user_gates_inline_to_the_gates_they_spell_out(qs):
    # Toffoli from H, T, T-dagger and CX (a textbook identity, exact)
    src = """OPENQASM 2.0;
    qreg a[2]; qreg t[1];
    gate tof x, y, z {
      h z; cx y, z; tdg z; cx x, z; t z; cx y, z; tdg z; cx x, z; t y; t z; h z;
      cx x, y; t x; tdg y; cx x, y;
    }
    tof a[0], a[1], t[0];
    """
    n, parsed = qs.parse_qasm(src)
    assert n == 3 and len(parsed) == 15
    psi0 = _state(3, 1)
    ref = oracle.simulate(3, [W.Gate("CCX", (0, 1, 2))], psi0)
    assert np.allclose(oracle.simulate(3, parsed, psi0), ref, atol=1e-13)
    # CPHASE(l) from U1 and CX with nested definitions and parameter expressions
    src = """OPENQASM 2.0;
    qreg q[2];
    gate half(l) x { u1(l/2) x; }
    gate mycu1(lam) c, t { half(lam) c; cx c, t; u1(-lam/2) t; cx c, t; half(2*lam/2) t; }
    mycu1(0.7*pi) q[0], q[1];
    """
    n, parsed = qs.parse_qasm(src)
    ref = oracle.simulate(2, [W.Gate("CP", (0, 1), (0.7 * np.pi,))], _state(2, 2))
    assert np.allclose(oracle.simulate(2, parsed, _state(2, 2)), ref, atol=1e-13)
    # exp(-i t/2 Z Z) from CX . RZ . CX (Sec. 5.1 ZZ term), ^ and unary minus in the angle
    src = "OPENQASM 2.0; qreg q[3]; gate zz(t) a, b { cx a, b; rz(t) b; cx a, b; } zz(-2^-1*sin(0.3)) q[2], q[0];"
    n, parsed = qs.parse_qasm(src)
    th = -0.5 * np.sin(0.3)
    ref = oracle.simulate(3, [W.Gate("RZZ", (2, 0), (th,))], _state(3, 3))
    assert np.allclose(oracle.simulate(3, parsed, _state(3, 3)), ref, atol=1e-13)
    # U and CX primitives; the textual qelib1 form of rz (u1) differs from RZ by a global phase only
    src = "OPENQASM 2.0; qreg q[1]; gate myrz(p) a { U(0, 0, p) a; } myrz(1.1) q[0];"
    _, parsed = qs.parse_qasm(src)
    assert _same_up_to_phase(oracle.simulate(1, parsed, _state(1, 4)),
                             oracle.simulate(1, [W.Gate("RZ", (0,), (1.1,))], _state(1, 4)))


def test_cu3_is_controlled_u3(qs):
    # controlled-U3 = diag(I, U3): the importer spells it with RZ, RY, CX and P, exactly
    from oracle import gates as G
    for t, p, l, c, tg in ((0.3, 1.1, -0.7, 2, 0), (2.5, -2.0, 0.4, 0, 1), (np.pi, 0.0, np.pi / 3, 1, 2)):
        n, parsed = qs.parse_qasm(f"OPENQASM 2.0; qreg q[3]; cu3({t!r}, {p!r}, {l!r}) q[{c}], q[{tg}];")
        psi0 = _state(3, 9)
        want = psi0.reshape(2, 2, 2).copy()   # axes: qubits 0, 1, 2
        sl = [slice(None)] * 3
        sl[c] = 1
        sub = want[tuple(sl)]                  # the control = 1 half, axes in qubit order without c
        ax = [q for q in range(3) if q != c].index(tg)
        want[tuple(sl)] = np.moveaxis(np.tensordot(G.matrix("U3", (t, p, l)), sub, axes=([1], [ax])), 0, ax)
        assert np.allclose(oracle.simulate(3, parsed, psi0), want.reshape(-1), atol=1e-14)
    # a program's own cu3 definition takes precedence
    _, parsed = qs.parse_qasm("OPENQASM 2.0; qreg q[2]; gate cu3(a, b, c) x, y { cx x, y; } cu3(1, 2, 3) q[0], q[1];")
    assert [g.kind for g in parsed] == ["CX"]


def test_c3x_c4x_are_multi_controlled_x(qs):
    # X on the last qubit where all the others are 1, exactly, with no ancilla
    for name, k, order in (("c3x", 3, (4, 0, 2, 1)), ("c4x", 4, (5, 1, 3, 0, 2))):
        n = k + 2
        _, parsed = qs.parse_qasm(f"OPENQASM 2.0; qreg q[{n}]; {name} " + ", ".join(f"q[{i}]" for i in order) + ";")
        psi0 = _state(n, k)
        want = psi0.copy()
        ctrl, tgt = order[:-1], order[-1]
        for x in range(2 ** n):
            if all((x >> (n - 1 - c)) & 1 for c in ctrl) and not (x >> (n - 1 - tgt)) & 1:
                y = x | (1 << (n - 1 - tgt))
                want[x], want[y] = psi0[y], psi0[x]
        assert np.allclose(oracle.simulate(n, parsed, psi0), want, atol=1e-14)


def test_sxdg_is_the_inverse_of_sx(qs):
    from oracle import gates as G
    _, parsed = qs.parse_qasm("OPENQASM 2.0; qreg q[2]; sxdg q[1]; sx q[1]; sxdg q[0];")
    psi0 = _state(2, 6)
    want = psi0.reshape(2, 2).copy()
    want = np.tensordot(G.matrix("SX", ()).conj().T, want, axes=([1], [0]))   # sxdg on qubit 0
    assert np.allclose(oracle.simulate(2, parsed, psi0), want.reshape(-1), atol=1e-14)


def test_registers_broadcast_and_statements_skipped(qs):
    src = """OPENQASM 2.0;
    include "qelib1.inc";   // line comment
    /* block
       comment */
    qreg a[3];
    qreg b[3];
    creg c[6];
    creg d[3];
    h a;
    cx a, b;
    rz(pi/4) b[1];
    barrier a, b;
    swap a[0], b;
    measure a[0] -> c[0];
    measure b -> d;
    """
    n, parsed = qs.parse_qasm(src)
    assert n == 6
    want = [("H", (0,)), ("H", (1,)), ("H", (2,)), ("CX", (0, 3)), ("CX", (1, 4)), ("CX", (2, 5)), ("RZ", (4,)),
            ("SWAP", (0, 3)), ("SWAP", (0, 4)), ("SWAP", (0, 5))]
    assert [(g.kind, tuple(g.wires)) for g in parsed] == want
    assert parsed[6].params == (np.pi / 4,)
    # a program with no gates
    n, parsed = qs.parse_qasm("OPENQASM 2.0; qreg q[4];")
    assert n == 4 and parsed == []


@pytest.mark.parametrize("src,status,line", [
    ("qreg q[4]; rc3x q[0], q[1], q[2], q[3];", 2, 1),                      # not in the gate set
    ("qreg q[4]; c3x q[0], q[1], q[2];", 1, 1),                               # c3x qubit count
    ("qreg q[2]; cu3(1, 2) q[0], q[1];", 1, 1),                               # cu3 parameter count
    ("qreg q[2];\nh q[2];", 1, 2),                                            # index out of range
    ("qreg q[2];\n\ncx q[1], q[1];", 1, 3),                                   # repeated qubit
    ("qreg q[2]; creg c[2]; measure q -> c;\nh q[0];", 2, 2),               # gate after a measurement
    ("qreg q[2] h q[0];", 1, 1),                                              # syntax
    ("qreg q[2]; reset q[0];", 2, 1),                                         # not unitary
    ("qreg q[2]; creg c[1]; if (c == 1) x q[0];", 2, 1),
    ("qreg q[2]; opaque g a; g q[0];", 2, 1),
    ('include "other.inc"; qreg q[1];', 2, 1),
    ("OPENQASM 3.0; qreg q[1];", 2, 1),
    ("qreg q[2]; qreg q[3];", 1, 1),                                          # declared twice
    ("qreg a[2]; qreg b[3]; cx a, b;", 1, 1),                                 # register sizes differ
    ("qreg q[2]; rx q[0];", 1, 1),                                            # parameter count
    ("qreg q[2]; rx(0.1) q;\nrx(0.1, 2) q[0];", 1, 2),
    ("qreg q[3]; ccx q[0], q[1];", 1, 1),                                     # qubit count
    ("qreg q[1]; rx(foo) q[0];", 1, 1),                                       # unknown name
    ("qreg q[1]; gate g a { h b; } g q[0];", 1, 1),                           # not an argument
    ("qreg q[1]; gate g a { g2 a; } gate g2 a { h a; } g q[0];", 1, 1),       # used before its definition
    ("qreg q[1]; gate U a { h a; }", 1, 1),                                   # primitive redefined
    ("creg c[1];", 1, 1),                                                     # no qreg
    ("qreg q[40]; qreg r[30];", 2, 1),                                        # more than 63 qubits
    ("qreg q[1]; /* open", 1, 1),
])
def test_errors_name_status_and_line(qs, src, status, line):
    with pytest.raises(qs.QsError) as e:
        qs.parse_qasm(src)
    assert e.value.status == status
    assert f"line {line}:" in str(e.value)


def test_null_arguments_are_rejected(qs):
    import ctypes
    arr = ctypes.POINTER(qs.QsGate)()
    ng, nq = ctypes.c_size_t(0), ctypes.c_int(0)
    assert qs._lib.qs_qasm_parse(None, ctypes.byref(arr), ctypes.byref(ng), ctypes.byref(nq)) == qs.QS_ERR_INVALID_ARG
    assert qs._lib.qs_qasm_parse(b"qreg q[1];", None, ctypes.byref(ng), ctypes.byref(nq)) == qs.QS_ERR_INVALID_ARG
    qs._lib.qs_qasm_free(None)


def test_imported_circuits_fuse_like_native_ones(qs):
    # GHZ / cat state: the CNOT chain is one gather pass (App. B.1)
    for n in (16, 22):
        src = f"OPENQASM 2.0;\ninclude \"qelib1.inc\";\nqreg q[{n}];\ncreg c[{n}];\nh q[0];\n"
        src += "".join(f"cx q[{i}], q[{i + 1}];\n" for i in range(n - 1))
        src += "barrier q;\nmeasure q -> c;\n"
        nq, parsed = qs.parse_qasm(src)
        txt_imp, p_imp = qs.plan_describe(nq, parsed)
        txt_nat, p_nat = qs.plan_describe(n, W.ghz_gates(n))
        assert p_imp == p_nat and txt_imp == txt_nat
        assert sum(1 for l in txt_imp.splitlines() if l.startswith(("GATHER", "PERM"))) == 1
    # QFT written with cu1 and swaps plans exactly as the generator's QFT
    n = 20
    _, parsed = qs.parse_qasm(to_qasm(n, W.qft_gates(n)))
    assert qs.plan_describe(n, parsed) == qs.plan_describe(n, W.qft_gates(n))
