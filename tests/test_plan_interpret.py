"""Fused plans checked on the host, pass by pass, against the oracle.

A C++ program links the planner, builds the plan the executor would run
(tile passes with sweeps, micro-ops, diagonal tables, count tables, QFT
ladders, dense blocks in FP32 / 3xTF32 / BF16 constant layouts; permutation
and gather passes), and interprets every pass on a complex128 state by the
contracts the pass descriptors document, checking their structural
invariants (tile and sweep bits, tensor-copy boxes, swizzled offsets,
constant bounds and alignment) on the way.  The final state must match the
complex128 oracle's gate-by-gate evolution of the same seeded input.  Batches
of parameter vectors run as the executor runs them: one plan per item, merged
into one plan with per-item constants and a batch coordinate in the tensor
copies.

Tolerances: constants are complex64 (relative error 2^-24 per entry), so a
plan of a few hundred ops drifts by at most ~1e-5 relative (L2); 1e-4 is
asserted.  BF16 dense blocks round U and X to 8-bit mantissas (2^-9 relative
per block), so plans with them are held to 3e-2, enough to expose a wrong
operand layout (an O(1) error)."""
import numpy as np
import pytest

import oracle
import plan_host
import workloads as W


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__._build_lib_module().build()
    import paper_2609_19147_gb300 as m
    return m


def _heisenberg(n, rng, rounds=2):
    g = []
    for _ in range(rounds):
        for b in range(n - 1):
            t = float(rng.uniform(-1, 1))
            g += [W.Gate("RXX", (b, b + 1), (t,)), W.Gate("RYY", (b, b + 1), (t,)), W.Gate("RZZ", (b, b + 1), (t,))]
        g += [W.Gate("RZ", (q,), (float(rng.uniform(-1, 1)),)) for q in range(n)]
    return g


def _zz_random_angles(n, rng):
    g = [W.Gate("H", (q,)) for q in range(n)]
    for _ in range(3 * n):
        u, v = (int(x) for x in rng.choice(n, size=2, replace=False))
        g.append(W.Gate("RZZ", (u, v), (float(rng.uniform(-3, 3)),)))
    g += [W.Gate("RX", (q,), (0.3,)) for q in range(n)]
    return g


def _param_layers(n, layers):
    """Layers of parameterised RX / RY / RZ, RZZ and CP (angles from a vector)."""
    g, k = [], 0
    for _ in range(layers):
        for q in range(n):
            g.append(W.Gate(("RX", "RY", "RZ")[q % 3], (q,), (0.0,), None, k))
            k += 1
        for q in range(0, n - 1, 2):
            g.append(W.Gate("RZZ", (q, q + 1), (0.0,), None, k))
            k += 1
        for q in range(1, n - 1, 2):
            g.append(W.Gate("CP", (q, q + 1), (0.0,), None, k))
            k += 1
    return g, k


def _u2_branch_layers(n, rng, layers=6):
    """U(2) layers split by CZ ladders whose matrices reach every branch of the
    phases-rotation-phases factorisation: Haar, diagonal (s = 0), anti-diagonal
    (c = 0), |c| > |s|, |s| > |c|, |c| = |s|."""
    gl = []
    for layer in range(layers):
        for q in range(n):
            kind = (q + layer) % 6
            if kind == 0:
                m = W.haar_u2(rng)
            else:
                th = {1: 0.0, 2: np.pi / 2, 3: 0.3, 4: 1.2, 5: np.pi / 4}[kind]
                a, b, d = rng.uniform(0.0, 2.0 * np.pi, 3)
                m = (np.diag(np.exp(1j * np.array([a, b]))) @ np.array([[np.cos(th), -np.sin(th)],
                                                                         [np.sin(th), np.cos(th)]])
                     @ np.diag([1.0, np.exp(1j * d)]))
            gl.append(W.Gate("U", (q,), (), m))
        gl += [W.Gate("CZ", (q, q + 1)) for q in range(n - 1)]
    return gl


def _cases():
    """(name, n, gates, (T, L, R, dense_prec, block_qubits)[, params (B x P)])"""
    rng = np.random.default_rng(23)
    out = []
    # random circuits over the whole vocabulary, several tile shapes and group sizes
    shapes = [(0, 0, 0), (8, 4, 5), (8, 2, 3), (7, 3, 4), (6, 1, 2), (9, 4, 1), (10, 3, 5)]
    for i, n in enumerate((9, 10, 11, 12)):
        for j, sh in enumerate(shapes):
            if (i + j) % 2 == 0:
                out.append((f"random n={n} {sh}", n, W.random_circuit(n, 90, 300 + 10 * i + j), sh + (0, 0)))
    # structured families at n = 14 (several tiles per pass)
    n = 14
    tf = W.tfim_gates(n, 4, 0.1, 1.0, W.tfim_fields(n, 3), order=2)
    qaoa = W.qaoa_gates(n, W.random_regular3_graph(n, rng), [0.4, 1.1], [0.7, 0.2])
    for sh in ((12, 4, 4), (13, 4, 5), (13, 4, 4), (9, 3, 3), (0, 0, 0)):
        out.append((f"tfim {sh}", n, tf, sh + (0, 0)))
        out.append((f"qaoa {sh}", n, qaoa, sh + (0, 0)))
    for sh in ((13, 4, 5), (12, 4, 4), (10, 2, 3), (0, 0, 0)):
        out.append((f"qft {sh}", n, W.qft_gates(n, swaps=True), sh + (0, 0)))
    out.append(("suite", 13, W.suite28_gates(13, 2, 5), (12, 4, 4, 0, 0)))
    out.append(("suite", 13, W.suite28_gates(13, 2, 6), (13, 4, 5, 0, 0)))
    out.append(("ghz + ladder", 12, W.ghz_gates(12) + W.cnot_ladder(12) + W.wht_gates(12), (10, 4, 4, 0, 0)))
    out.append(("controlled", 9, W.random_circuit(9, 80, 77, kinds=["CCX", "CSWAP", "CX", "CH", "CRY", "CY", "H"]),
                (7, 2, 5, 0, 0)))
    out.append(("heisenberg", 12, _heisenberg(12, rng), (10, 4, 5, 0, 0)))
    out.append(("u2 branches r5", 12, _u2_branch_layers(12, rng), (10, 4, 5, 0, 0)))
    out.append(("u2 branches r4", 12, _u2_branch_layers(12, rng), (9, 3, 4, 0, 0)))
    out.append(("zz random angles", 12, _zz_random_angles(12, rng), (9, 4, 4, 0, 0)))
    out.append(("zz random angles r5", 12, _zz_random_angles(12, rng), (12, 4, 5, 0, 0)))
    # dense blocks in every precision and block size
    for prec in (1, 2, 3):
        for k in (3, 4, 5):
            out.append((f"dense p={prec} k={k} random", 11, W.random_circuit(11, 80, 900 + 3 * prec + k),
                        (9, 4, 5, prec, k)))
        out.append((f"dense p={prec} tfim", 14, tf, (13, 4, 5, prec, 5)))
    # two-qubit diagonals spelled out as CX . diagonal . CX (folded by the detector)
    out.append(("spelled qft", 14, W.spell_out_2q(W.qft_gates(14)), (13, 4, 5, 0, 0)))
    out.append(("spelled tfim", 14, W.spell_out_2q(tf), (12, 4, 4, 0, 0)))
    out.append(("spelled qaoa", 14, W.spell_out_2q(qaoa), (13, 4, 5, 0, 0)))
    for n, sh in ((10, (8, 4, 4)), (11, (9, 3, 5)), (12, (0, 0, 0))):
        out.append((f"cx sandwiches n={n}", n, W.cx_sandwich_circuit(n, 60, 700 + n), sh + (0, 0)))
    out.append(("cx sandwiches dense", 11, W.cx_sandwich_circuit(11, 60, 720), (9, 4, 5, 2, 4)))
    # long circuits on states that fit one tile: every pass ends at the sweep or
    # micro-op limit, and the ops it has no room for must carry over
    out.append(("tfim 12q 40 steps", 12, W.tfim_gates(12, 40, 0.05, 1.0, W.tfim_fields(12, 11), order=2),
                (0, 0, 0, 0, 0)))
    out.append(("tfim 13q 20 steps r4", 13, W.tfim_gates(13, 20, 0.05, 1.0, 0.7, order=2), (13, 4, 4, 0, 0)))
    out.append(("random 10q 600 gates", 10, W.random_circuit(10, 600, 77), (10, 4, 5, 0, 0)))
    out.append(("qaoa 12q p=12", 12, W.qaoa_gates(12, W.random_regular3_graph(12, rng), list(np.linspace(0.1, 1, 12)),
                                                 list(np.linspace(1, 0.1, 12))), (0, 0, 0, 0, 0)))
    # per-gate plans (the baseline path: one launch per gate over its subspace)
    for n in (3, 8, 11):
        out.append((f"pergate random n={n}", n, W.random_circuit(n, 120, 1200 + n), (0, 0, 0, 0, 0, 1)))
    out.append(("pergate qft", 12, W.qft_gates(12), (0, 0, 0, 0, 0, 1)))
    out.append(("pergate tfim", 12, W.tfim_gates(12, 3, 0.1, 1.0, 0.7, order=2), (0, 0, 0, 0, 0, 1)))
    out.append(("pergate sandwiches", 10, W.cx_sandwich_circuit(10, 40, 1300), (0, 0, 0, 0, 0, 1)))
    out.append(("pergate vqe batch", 10, W.vqe_ansatz_gates(10, 2), (0, 0, 0, 0, 0, 1), W.vqe_params(10, 2, 3, 9)))
    # batches of parameter vectors (per-item constants in one merged plan)
    vqe = W.vqe_ansatz_gates(12, 3)
    for sh in ((12, 4, 4), (10, 3, 5), (0, 0, 0)):
        out.append((f"vqe batch {sh}", 12, vqe, sh + (0, 0), W.vqe_params(12, 3, 4, 8)))
    pl, k = _param_layers(11, 3)
    out.append(("param layers batch", 11, pl, (9, 4, 4, 0, 0), rng.uniform(-3, 3, size=(3, k))))
    out.append(("param layers batch dense", 11, pl, (9, 4, 5, 1, 4), rng.uniform(-3, 3, size=(2, k))))
    return out


def test_plans_interpreted_on_host_match_oracle(tmp_path, qs):
    if not plan_host.available():
        pytest.skip("needs g++ and the CUDA headers")
    cases = _cases()
    psi0s, expect = [], []
    for i, case in enumerate(cases):
        name, n, gl = case[:3]
        params = case[4] if len(case) > 4 else np.zeros((1, 0))
        B, P = params.shape
        rng = np.random.default_rng(1000 + i)
        psi0 = rng.standard_normal((B, 2 ** n)) + 1j * rng.standard_normal((B, 2 ** n))
        psi0 /= np.linalg.norm(psi0, axis=1, keepdims=True)
        psi0s.append(psi0)
        expect.append(np.stack([oracle.simulate(n, gl, psi0[b].copy(), theta=params[b] if P else None)
                                for b in range(B)]))
    res = plan_host.interpret(qs, cases, str(tmp_path), psi0s)
    micro = np.zeros(13, dtype=np.int64)
    dense = np.zeros(3, dtype=np.int64)
    kinds = {"perm": 0, "gather": 0, "tma": 0, "rows": 0, "swz": 0, "pergate": 0}
    for i, case in enumerate(cases):
        name, n, gl, cfg = case[:4]
        got, f = res[i]
        if len(case) > 4 and case[4].shape[0] > 1 and len(cfg) < 6:
            assert f["merged"] == 1, (name, "item plans did not merge")
        for k in kinds:
            kinds[k] += f[k]
        micro += np.array(f["micro"])
        dense += np.array(f["dense"])
        err = np.max(np.linalg.norm(got - expect[i], axis=1) / np.linalg.norm(expect[i], axis=1))
        tol = 3e-2 if cfg[3] == 3 else 1e-4
        assert err < tol, (name, cfg, err)
    # every pass type, copy form and micro-op kind was exercised
    assert all(v > 0 for v in kinds.values()), kinds
    assert all(micro > 0), micro
    assert all(dense > 0), dense
