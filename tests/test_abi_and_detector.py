"""CPU tests of the C-ABI library: it loads, exports every symbol include/qs.h
declares, validates arguments without touching a GPU, and its fusion detector
produces the expected pass structure (Sec. 5.1-5.2 pass-count arguments;
App. A H-layer accounting)."""
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__._build_lib_module().build()
    import paper_2609_19147_gb300 as m
    return m


def _header_functions():
    src = open(os.path.join(ROOT, "include", "qs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(qs):
    import ctypes
    lib = ctypes.CDLL(qs.LIB_PATH)
    declared = _header_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(qs.EXPORTED)


def test_version_and_no_error(qs):
    assert "sm_103a" in qs.version()


def _status(qs, n, gates):
    try:
        qs.plan_describe(n, gates)
        return qs.QS_OK
    except qs.QsError as e:
        return e.status


def test_validation_rejects_bad_gates(qs):
    assert _status(qs, 4, [W.Gate("CX", (1, 1))]) == qs.QS_ERR_INVALID_ARG      # duplicate wire
    assert _status(qs, 4, [W.Gate("H", (4,))]) == qs.QS_ERR_INVALID_ARG         # out of range
    assert _status(qs, 4, [W.Gate("H", (-1,))]) == qs.QS_ERR_INVALID_ARG
    assert _status(qs, 40, [W.Gate("H", (0,))]) == qs.QS_ERR_UNSUPPORTED        # n > 33
    g = qs.CGates([W.Gate("H", (0,))])
    g.arr[0].nw = 2                                                              # wrong arity
    assert _status(qs, 4, g) == qs.QS_ERR_INVALID_ARG
    g = qs.CGates([W.Gate("H", (0,))])
    g.arr[0].kind = 999
    assert _status(qs, 4, g) == qs.QS_ERR_INVALID_ARG
    g = qs.CGates([W.Gate("U", (0,), (), np.eye(2))])
    g.arr[0].dense = None
    assert _status(qs, 4, g) == qs.QS_ERR_INVALID_ARG
    g = qs.CGates([W.Gate("RX", (0,), (np.nan,))])
    assert _status(qs, 4, g) == qs.QS_ERR_INVALID_ARG
    g = qs.CGates([W.Gate("U", (0,), (), np.array([[np.inf, 0], [0, 1]]))])   # non-finite matrix entry
    assert _status(qs, 4, g) == qs.QS_ERR_INVALID_ARG
    g = qs.CGates([W.Gate("CZ", (0, 1))])
    g.arr[0].kind = 1000                                                         # the detector's internal kind
    assert _status(qs, 4, g) == qs.QS_ERR_INVALID_ARG
    # parameter index without a parameter vector
    assert _status(qs, 4, [W.Gate("RX", (0,), (0.0,), None, 0)]) == qs.QS_ERR_INVALID_ARG


def _passes(qs, n, gates, **kw):
    return qs.plan_describe(n, gates, **kw)


def test_qft_stages_fuse_into_few_passes(qs):
    # every stage (H + its CP ladder) is recognised: 30 stages -> 3 tile passes
    # plus one permutation pass for the final swaps (bit reversal)
    text, p = _passes(qs, 30, W.qft_gates(30, swaps=True))
    assert p == 4
    assert text.count("QFT=") == 3 and "PERM" in text
    assert sum(int(x) for x in re.findall(r"QFT=(\d+)", text)) == 29   # last stage has no ladder
    text, p = _passes(qs, 30, W.qft_gates(30, swaps=False))
    assert p == 3 and "PERM" not in text
    _, p = _passes(qs, 30, W.qft_gates(30, swaps=True), mode="pergate")
    assert p == 480


def test_u2_layers_become_phase_rotation_phase_sweeps(qs):
    # a sweep whose only op is a layer of general 2x2 unitaries on all its
    # group bits is planned as phases, rotations, phases (one ZYZ op per sweep)
    rng = np.random.default_rng(3)
    n = 20
    gl = [W.Gate("U", (q,), (), W.haar_u2(rng)) for q in range(n)]
    text, _ = _passes(qs, n, gl)
    zyz = [int(x) for x in re.findall(r"ZYZ=(\d+)", text)]
    assert sum(zyz) >= 4 and all(int(x) == 0 for x in re.findall(r" U1=(\d+)", text)), text
    # the factorisation holds for unitary matrices only: a scaled layer keeps
    # the general 2x2 form
    text, _ = _passes(qs, n, [W.Gate("U", (q,), (), 0.9 * W.haar_u2(rng)) for q in range(n)])
    assert all(int(x) == 0 for x in re.findall(r"ZYZ=(\d+)", text)), text
    assert sum(int(x) for x in re.findall(r" U1=(\d+)", text)) == n, text


def _tile_bit_sets(text):
    out = []
    for m in re.finditer(r"TILE T=\d+ L=\d+ hb=\[([\d,]*)\] tma=(\d)", text):
        out.append(([int(x) for x in m.group(1).split(",") if x], m.group(2) == "1"))
    return out


def test_layer_order_for_locality_is_chosen_by_cost(qs):
    # 30q Trotter steps: the real-rotation layers are ordered so that no pass
    # keeps six or more 2 MB-page bits (index bit 18 and up) reaching bit 27
    # or above, with the same pass count as the stream order
    n = 30
    gl = W.tfim_gates(n, 20, 0.05, 1.0, W.tfim_fields(n, 3), order=2)
    kw = dict(tile_qubits=13, low_qubits=4, group_qubits=5)
    text, p = _passes(qs, n, gl, **kw)
    assert p == 41
    for hb, tma in _tile_bit_sets(text):
        assert tma
        assert not (sum(b >= 18 for b in hb) >= 6 and max(hb) >= 27), hb
    # Heisenberg chains: the reordered layers would fragment passes past one
    # tensor copy; the stream order is kept (no row-by-row passes)
    text, _ = _passes(qs, n, dict(W.sweep_workloads(n))["heisenberg_chain"], **kw)
    assert all(tma for _, tma in _tile_bit_sets(text))
    # below 2^28 amplitudes the stream order stands
    n = 25
    text25, _ = _passes(qs, n, W.tfim_gates(n, 4, 0.05, 1.0, W.tfim_fields(n, 3), order=2), **kw)
    assert _tile_bit_sets(text25)[0][0] == list(range(16, 25))


def test_default_shape_takes_5_bit_groups_for_layer_plans(qs):
    # on a tie in passes the planner takes 13-bit tiles with 5-bit groups for
    # layer plans (uncontrolled one-qubit layers and diagonals) and QFT
    # stages, and keeps 4-bit groups for circuits with controlled ops
    fams = dict(W.sweep_workloads(25))
    for name in ("tfim_2nd_order", "heisenberg_chain", "qaoa_ring", "variational_ansatz", "qft"):
        text, _ = _passes(qs, 25, fams[name])
        assert set(re.findall(r" R=(\d)", text)) == {"5"}, (name, text)
    for name in ("random_circuit", "quantum_walk", "long_range_ising"):
        text, _ = _passes(qs, 25, fams[name])
        assert "5" not in set(re.findall(r" R=(\d)", text)), (name, text)


def test_h_layer_pass_count_app_a(qs):
    # App. A: radix-4 Walsh takes ceil(25/4) = 7 passes; tiles of 13 qubits take 3
    text, p = _passes(qs, 25, W.wht_gates(25))
    assert p == 3
    _, p = _passes(qs, 25, W.wht_gates(25), tile_qubits=6, low_qubits=2)
    assert p == 6


def test_gf2_runs_become_one_pass(qs):
    text, p = _passes(qs, 24, W.cnot_ladder(24))
    assert p == 1 and "GATHER" in text
    # SWAP run -> permutation pass
    text, p = _passes(qs, 24, [W.Gate("SWAP", (i, 23 - i)) for i in range(12)])
    assert p == 1 and "PERM" in text
    # GHZ: H then one gather for the 23-gate CNOT chain (Sec. 5.1: 24-gate chain -> one pass)
    text, p = _passes(qs, 24, W.ghz_gates(24))
    assert p == 2 and "GATHER" in text


def test_diagonal_runs_fuse(qs):
    rng = np.random.default_rng(0)
    gl = [W.Gate("RZZ", (b, b + 1), (float(rng.uniform(0, 6.28)),)) for b in range(27)]
    text, p = _passes(qs, 28, gl)
    assert p == 1 and "DIAG=1" in text
    # the paper's long-range Ising layer: 300 all-to-all bonds at 25 qubits, one pass
    gl = [W.Gate("RZZ", (i, j), (0.1 / (j - i),)) for i in range(25) for j in range(i + 1, 25)]
    assert len(gl) == 300
    _, p = _passes(qs, 25, gl)
    assert p == 1


def test_identity_windows_vanish_and_small_angles_survive(qs):
    # H H and X X cancel symbolically (Sec. 5.2 exact collapse); RZ(1e-6) is kept (rtol = 0)
    text, p = _passes(qs, 10, [W.Gate("H", (3,)), W.Gate("H", (3,)), W.Gate("X", (2,)), W.Gate("X", (2,))])
    assert p == 0
    text, p = _passes(qs, 10, [W.Gate("RZ", (3,), (1e-6,))])
    assert p == 1 and "DIAG=1" in text


def test_no_cross_family_merge_for_ladder_heisenberg(qs):
    # interleaved XX / YY / ZZ on the same bonds must keep their order: the
    # detector may not reorder non-commuting terms (Sec. 5.2, App. B ladder)
    n = 8
    gl = []
    for b in range(n - 1):
        gl += [W.Gate("RXX", (b, b + 1), (0.3,)), W.Gate("RYY", (b, b + 1), (0.3,)),
               W.Gate("RZZ", (b, b + 1), (0.3,))]
    text, p = _passes(qs, n, gl)
    assert p >= 1   # correctness of the order is checked on the GPU against the oracle


def test_tfim_trotter_steps_pack(qs):
    h = W.tfim_fields(30, 3)
    gl = W.tfim_gates(30, 10, 0.05, 1.0, h, order=2)
    _, p = _passes(qs, 30, gl)
    _, pg = _passes(qs, 30, gl, mode="pergate")
    assert pg == len(gl) == 10 * (29 * 2 + 30)
    assert p <= 3 * 10          # <= 3 HBM passes per Strang step


# --- dense k-qubit blocks (qs_opts dense_prec / block_qubits) -----------------
def test_dense_blocks_tfim_plan(qs):
    # 30q TFIM, 100 Strang steps: per step the X layer and the in-cell ZZ bonds
    # become 7 dense blocks (cells of 4-5 bits filling the 13-bit tile windows)
    # and the 6 cross-cell bonds stay diagonal; the dense plans take no more
    # HBM passes than the structured one
    h = W.tfim_fields(30, 3)
    gl = W.tfim_gates(30, 100, 0.05, 1.0, h, order=2)
    _, p0 = _passes(qs, 30, gl)
    for d in ("fp32", "tf32x3", "bf16"):
        text, p = _passes(qs, 30, gl, dense=d)
        blocks = sum(int(m) for m in re.findall(r"DENSE=(\d+)", text))
        assert blocks == 7 * 100, (d, blocks)
        assert p <= p0, (d, p, p0)


def test_dense_blocks_general_circuits_plan(qs):
    gl = W.random_circuit(14, 300, 4242)
    for k in (3, 4, 5):
        text, p = _passes(qs, 14, gl, dense="tf32x3", block_qubits=k)
        assert "DENSE=" in text and p >= 1
    # a state smaller than a 13-bit tile: the tile is the whole state
    text, _ = _passes(qs, 6, W.random_circuit(6, 60, 1), dense="bf16")
    assert "T=6" in text and "DENSE=" in text


def test_dense_options_validated(qs):
    import ctypes
    gl = [W.Gate("H", (0,))]
    for k in (1, 2, 6, -1):
        with pytest.raises(qs.QsError) as e:
            qs.plan_describe(8, gl, dense="fp32", block_qubits=k)
        assert e.value.status == qs.QS_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        qs.plan_describe(8, gl, dense="fp64")
    cg = qs.CGates(gl)
    o = qs._opts()
    o.dense_prec = 9
    assert qs._lib.qs_plan_describe(8, cg.arr, cg.n, ctypes.byref(o), None, 0, None) == qs.QS_ERR_INVALID_ARG


def test_pauli_pair_layers_are_basis_conjugated(qs):
    # a run of RXX (or RYY) gates becomes 1q layers around one ZZ diagonal:
    # no 4x4 ops remain; a lone RXX stays a 4x4 op
    n = 16
    for kind in ("RXX", "RYY"):
        gl = [W.Gate(kind, (i, i + 1), (0.2 + 0.01 * i,)) for i in range(n - 1)]
        text, p = _passes(qs, n, gl)
        assert sum(int(m) for m in re.findall(r"U2=(\d+)", text)) == 0, text
        assert sum(int(m) for m in re.findall(r"DIAG=(\d+)", text)) >= 1
    text, _ = _passes(qs, n, [W.Gate("RXX", (3, 9), (0.4,))])
    assert sum(int(m) for m in re.findall(r"U2=(\d+)", text)) == 1


def test_uniform_pair_sums_become_count_lookups(qs):
    # uniform-angle RZZ chains (TFIM, including the S phases of conjugated RX
    # layers), uniform CZ rings and uniform RZZ on a random graph take the
    # count-table diagonal; random-angle ZZ bonds keep the factored tables
    n = 30
    tf = W.tfim_gates(n, 4, 0.05, 1.0, W.tfim_fields(n, 3), order=2)
    text, _ = _passes(qs, n, tf)
    d = sum(int(m) for m in re.findall(r" DIAG=(\d+)", text))
    assert sum(int(m) for m in re.findall(r"DIAGC=(\d+)", text)) == d > 0, text
    ring = [W.Gate("CZ", (b, (b + 1) % 20)) for b in range(20)] + [W.Gate("H", (q,)) for q in range(20)]
    assert "DIAGC=" in _passes(qs, 20, ring)[0]
    g = W.random_regular3_graph(18, np.random.default_rng(4))
    gl = [W.Gate("RZZ", (u, v), (0.3,)) for u, v in g] + [W.Gate("RX", (q,), (0.2,)) for q in range(18)]
    assert "DIAGC=" in _passes(qs, 18, gl)[0]
    rng = np.random.default_rng(2)
    rz = [W.Gate("RZZ", (b, b + 1), (float(rng.uniform(0, 6)),)) for b in range(27)]
    assert "DIAGC=" not in _passes(qs, 28, rz)[0]


def test_qaoa_cost_layers_and_tfim_pass_count(qs):
    # every cost layer of a QAOA circuit on a 3-regular graph is a count
    # lookup, and the 30q TFIM workload keeps its 201 HBM passes (100 Strang
    # steps: the light-cone fusion of consecutive steps)
    n = 20
    edges = W.random_regular3_graph(n, np.random.default_rng(9))
    gl = W.qaoa_gates(n, edges, [0.4, 0.7, 1.1, 0.2], [0.3, 0.5, 0.9, 1.3])
    text, _ = _passes(qs, n, gl)
    d = sum(int(m) for m in re.findall(r" DIAG=(\d+)", text))
    assert sum(int(m) for m in re.findall(r"DIAGC=(\d+)", text)) == d >= 4, text
    tf = W.tfim_gates(30, 100, 0.05, 1.0, W.tfim_fields(30, 3), order=2)
    assert _passes(qs, 30, tf)[1] == 201


def test_planner_fuzz_all_option_combinations(qs):
    # random circuits over the whole vocabulary, uniform-angle layers and
    # random graphs, planned under every tile shape / group size / dense
    # precision: the planner either succeeds with at least one pass for a
    # non-trivial circuit or rejects an invalid option with INVALID_ARG --
    # never another status (no internal scheduling failure)
    rng = np.random.default_rng(2024)
    shapes = [(0, 0, 0), (13, 4, 4), (13, 5, 5), (12, 4, 5), (12, 5, 4), (10, 3, 3), (8, 2, 2), (13, 4, 1)]
    precs = [None, "fp32", "tf32x3", "bf16"]
    for trial in range(200):
        n = int(rng.integers(2, 23))
        kind = trial % 3
        if kind == 0:
            gl = W.random_circuit(n, int(rng.integers(5, 120)), int(rng.integers(1 << 30)))
        elif kind == 1:
            th = float(rng.uniform(-3, 3))
            gl = [W.Gate("RY", (q,), (float(rng.uniform(0, 6)),)) for q in range(n)]
            gl += [W.Gate("RZZ", (b, b + 1), (th,)) for b in range(n - 1)]
            gl += [W.Gate("RZ", (q,), (0.3,)) for q in range(0, n, 2)]
            gl += [W.Gate("RX", (q,), (float(rng.uniform(0, 6)),)) for q in range(n)]
        else:
            m = n + (n & 1) if n >= 4 else 4
            edges = W.random_regular3_graph(m, rng)
            gl = W.qaoa_gates(m, edges, [0.5, 1.2], [0.3, 0.8])
            n = m
        t, lq, r = shapes[int(rng.integers(len(shapes)))]
        prec = precs[int(rng.integers(len(precs)))]
        try:
            text, passes = qs.plan_describe(n, gl, tile_qubits=t, low_qubits=lq, group_qubits=r, dense=prec)
        except qs.QsError as e:
            assert e.status == qs.QS_ERR_INVALID_ARG, (trial, n, t, lq, r, prec, str(e))
            continue
        assert passes >= 0 and text.startswith("FUSED"), (trial, text[:200])


def test_c_program_uses_the_abi(qs, tmp_path):
    # qs.h compiles as C11 and a C program links libqs.so and calls it (no GPU needed)
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("needs gcc")
    lib_dir = os.path.dirname(qs.LIB_PATH)
    exe = str(tmp_path / "c_abi_check")
    subprocess.check_call([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "cpp", "c_abi_check.c"), "-L", lib_dir, "-lqs",
                           "-Wl,-rpath," + lib_dir, "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr

