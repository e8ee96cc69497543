"""qs_qasm_parse on malformed and adversarial programs: random token and
byte mutations of valid programs, and inputs aimed at the parser's limits
(100k-deep parentheses, sign and power chains, definitions that expand to
2^60 calls or nest 200 deep, out-of-range sizes and indices, non-finite
angles, empty and truncated programs).  Every call must return a status
(QS_ERR_INVALID_ARG / QS_ERR_UNSUPPORTED with a line number) or valid
records; the fuzzing runs in a child process so that a crash fails the test
instead of the test run."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__._build_lib_module().build()


def test_parser_survives_fuzzing(built):
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([ROOT, HERE, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "qasm_fuzz_child.py"), "7", "1500"],
                       capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
    line = [l for l in r.stdout.splitlines() if l.startswith("FUZZ")][-1]
    stats = dict(kv.split("=") for kv in line.split()[1:])
    assert int(stats["ok"]) > 50 and int(stats["err"]) > 500, stats


def test_parser_mutation_fuzz_under_sanitizers(tmp_path):
    # the parser alone, in-process, under AddressSanitizer and UBSan
    import shutil
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    exe = str(tmp_path / "qasm_mutation_fuzz")
    csrc = os.path.join(ROOT, "paper_2609_19147_gb300", "csrc")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                        "-I", os.path.join(ROOT, "include"), "-I", csrc,
                        os.path.join(HERE, "cpp", "qasm_mutation_fuzz.cpp"), os.path.join(csrc, "qs_qasm.cpp"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no sanitizer runtime: " + r.stderr[-200:])
    out = subprocess.run([exe, "5", "6000"], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-1000:] + out.stderr[-3000:]
    ok, err = (int(kv.split("=")[1]) for kv in out.stdout.split())
    assert ok + err == 6000 and ok > 20

