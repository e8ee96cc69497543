"""Child process of test_qasm_fuzz.py: feeds qs_qasm_parse mutated and
adversarial programs and checks each call returns a status (a crash or hang
of this process fails the parent test).  Prints one summary line."""
import sys

import numpy as np


def main(seed: int, rounds: int):
    import paper_2609_19147_gb300 as qs
    rng = np.random.default_rng(seed)
    base = [
        'OPENQASM 2.0;\ninclude "qelib1.inc";\nqreg q[5];\nqreg r[3];\ncreg c[5];\n'
        'gate zz(t) a, b { cx a, b; rz(t) b; cx a, b; }\n'
        'gate lay(t, f) a, b { ry(f) a; zz(t*pi/2) a, b; u3(f, -t, 2^-1) b; }\n'
        'h q;\nlay(0.3, sin(0.2)) q[0], r[1];\ncx q[1], r[2];\ncu1(pi/4) q[2], q[3];\n'
        'barrier q, r;\nccx q[0], q[1], r[0];\nswap r[0], q[4];\nmeasure q -> c;\n',
        'OPENQASM 2.0;\nqreg a[4];\n/* c */ rx(-(1.5e-1)) a;\ncswap a[0], a[1], a[2];\nrzz(ln(2)) a[3], a[0];\n',
    ]
    vocab = ["OPENQASM", "2.0", "include", '"qelib1.inc"', "qreg", "creg", "gate", "opaque", "barrier",
             "measure", "reset", "if", "q", "r", "a", "b", "t", "[", "]", "(", ")", "{", "}", ";", ",", "->",
             "==", "+", "-", "*", "/", "^", "pi", "sin", "cos", "sqrt", "ln", "exp", "0", "1", "7", "1e308",
             "2.5", "h", "cx", "u3", "rz", "ccx", "zz", "lay", "U", "CX", "//", "/*", "*/", '"', "\n"]
    ok = err = 0
    gates_total = 0

    def run(src):
        nonlocal ok, err, gates_total
        try:
            n, g = qs.parse_qasm(src)
        except qs.QsError as e:
            assert e.status in (qs.QS_ERR_INVALID_ARG, qs.QS_ERR_UNSUPPORTED), e
            assert "line " in str(e), e
            err += 1
            return
        except UnicodeError:
            err += 1
            return
        assert 1 <= n <= 63
        for x in g:
            assert all(0 <= w < n for w in x.wires) and len(set(x.wires)) == len(x.wires)
            assert all(np.isfinite(p) for p in x.params)
        gates_total += len(g)
        ok += 1

    for _ in range(rounds):
        src = base[int(rng.integers(len(base)))]
        toks = src.replace("(", " ( ").replace(")", " ) ").replace(";", " ; ").replace(",", " , ").split(" ")
        for _ in range(int(rng.integers(1, 4))):
            op = int(rng.integers(4))
            k = int(rng.integers(len(toks)))
            if op == 0:
                del toks[k]
            elif op == 1:
                toks.insert(k, str(rng.choice(vocab)))
            elif op == 2:
                toks[k] = str(rng.choice(vocab))
            else:
                j = int(rng.integers(len(toks)))
                toks[k], toks[j] = toks[j], toks[k]
        run(" ".join(toks))
        # raw byte noise inside a valid program
        s = list(base[0])
        for _ in range(int(rng.integers(1, 6))):
            s[int(rng.integers(len(s)))] = chr(int(rng.integers(1, 127)))
        run("".join(s))
    # adversarial inputs: each must come back with an error status, quickly
    adv = [
        "qreg q[1]; rx(" + "(" * 100000 + "1" + ")" * 100000 + ") q[0];",
        "qreg q[1]; rx(" + "-" * 100000 + "1) q[0];",
        "qreg q[1]; rx(" + "2^" * 50000 + "2) q[0];",
        "qreg q[1]; rx(" + "sin(" * 50000 + "1" + ")" * 50000 + ") q[0];",
        "qreg q[1]; gate g0 a { barrier a; }\n" + "".join(
            f"gate g{i} a {{ g{i - 1} a; g{i - 1} a; }}\n" for i in range(1, 61)) + "g60 q[0];",
        "qreg q[1]; gate g0 a { h a; }\n" + "".join(
            f"gate g{i} a {{ g{i - 1} a; }}\n" for i in range(1, 200)) + "g199 q[0];",
        "qreg q[99999999999999999999];",
        "qreg q[2]; h q[99999999999999999999];",
        "qreg q[1]; rx(1e999) q[0];",
        "qreg q[1]; rx(sqrt(-1)) q[0];",
        "qreg q[1]; rx(ln(0)) q[0];",
        "qreg q[1]; rx(0/0) q[0];",
        "",
        ";" * 1000,
        "qreg q[1]; h q[0]" * 1000,
        "\x00qreg q[1];",
    ]
    for src in adv:
        try:
            qs.parse_qasm(src)
            raise AssertionError("accepted: " + src[:60])
        except qs.QsError as e:
            assert e.status in (qs.QS_ERR_INVALID_ARG, qs.QS_ERR_UNSUPPORTED), e
    print(f"FUZZ ok={ok} err={err} gates={gates_total} adversarial={len(adv)}", flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]), int(sys.argv[2]))
