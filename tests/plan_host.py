"""Runs the host plan interpreter (tests/cpp/plan_interpret_check.cpp) over a
list of cases and returns, per case, the final states and the interpreter's
pass / micro-op counts.  With QS_HOST_SANITIZE=1 in the environment the
interpreter and the planner are built with AddressSanitizer and UBSan.

A case is (name, n, gates, (T, L, R, dense_prec, block_qubits[, mode])[, params]),
mode 0 = fused (default) or 1 = per-gate, params a B x P array of parameter
vectors (one state per row)."""
import os
import shutil
import subprocess

import numpy as np

from gate_text import gate_lines

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def available():
    return shutil.which("g++") is not None and os.path.isdir("/usr/local/cuda/include")


def interpret(qs, cases, workdir, psi0s):
    """psi0s[i]: B x 2^n complex128 input states of case i, or None for a
    structure-only check (every invariant and the boxes of sampled tiles, no
    state: for sizes too large for the host).  Returns a list of (states
    B x 2^n or None, counts dict) in case order; raises AssertionError with the
    interpreter's message if a plan breaks an invariant."""
    lines = []
    for i, case in enumerate(cases):
        name, n, gl, cfg = case[:4]
        T, L, R, prec, blk = cfg[:5]
        mode = cfg[5] if len(cfg) > 5 else 0
        params = case[4] if len(case) > 4 else np.zeros((1, 0))
        B, P = params.shape
        if psi0s[i] is None:
            fin = fout = "-"
        else:
            fin, fout = os.path.join(workdir, f"in{i}.bin"), os.path.join(workdir, f"out{i}.bin")
            np.ascontiguousarray(psi0s[i], dtype=np.complex128).tofile(fin)
        text = gate_lines(qs, gl, pidx=True)
        lines.append(f"case {n} {T} {L} {R} {prec} {blk} {mode} {len(text)} {B} {P} {fin} {fout}")
        lines += text
        lines += [" ".join(repr(float(v)) for v in row) for row in params if P]
    src = os.path.join(workdir, "cases.txt")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    csrc = os.path.join(ROOT, "paper_2609_19147_gb300", "csrc")
    exe = os.path.join(workdir, "plan_interpret_check")
    # QS_HOST_SANITIZE=1: build the interpreter and the planner with AddressSanitizer and UBSan
    san = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"] \
        if os.environ.get("QS_HOST_SANITIZE") == "1" else ["-O2"]
    subprocess.check_call([shutil.which("g++")] + san + ["-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                           "-I", "/usr/local/cuda/include",
                           os.path.join(ROOT, "tests", "cpp", "plan_interpret_check.cpp"),
                           os.path.join(csrc, "qs_plan.cpp"), "-o", exe, "-lpthread"])
    out = subprocess.run([exe, src], capture_output=True, text=True, timeout=3000)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    rows = [l.split() for l in out.stdout.splitlines() if l.startswith("CASE")]
    assert len(rows) == len(cases)
    res = []
    for i, case in enumerate(cases):
        r = rows[i]
        counts = {k: int(v) for k, v in zip(r[2:20:2], r[3:20:2])}
        mi, di = r.index("micro"), r.index("dense")
        counts["micro"] = [int(x) for x in r[mi + 1:mi + 14]]
        counts["dense"] = [int(x) for x in r[di + 1:di + 4]]
        counts["pergate"] = int(r[r.index("pergate") + 1])
        if psi0s[i] is None:
            res.append((None, counts))
            continue
        shape = np.asarray(psi0s[i]).shape
        states = np.fromfile(os.path.join(workdir, f"out{i}.bin"), dtype=np.complex128).reshape(shape)
        res.append((states, counts))
    return res
