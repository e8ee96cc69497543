"""Planner fuzz on the host: random small circuits (the whole gate
vocabulary, CX . diagonal . CX blocks, TFIM, QFT tails) under random tile
shapes (tile bits 1..13, low bits 1..4, group sizes 1..5, including shapes the
planner must clamp), dense precisions and block sizes.  Every plan must build
(no 'could not place' internal errors), keep the interpreter's structural
invariants, and match the oracle: relative L2 <= 1e-4, or 6e-2 with BF16
blocks (8-bit mantissas, rounding accumulating over up to ~100 blocks)."""
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


def _cases(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for trial in range(count):
        n = int(rng.integers(1, 11))
        cfg = (int(rng.choice([0, 1, 2, 3, 5, 7, 9, 12, 13])), int(rng.choice([0, 1, 2, 3, 4])),
               int(rng.choice([0, 1, 2, 3, 4, 5])), int(rng.choice([0, 0, 0, 1, 2, 3])), int(rng.choice([0, 3, 4, 5])))
        mix = rng.random()
        if mix < 0.5:
            gl = W.random_circuit(n, int(rng.integers(1, 150)), int(rng.integers(1 << 30)))
        elif mix < 0.7 and n >= 2:
            gl = W.cx_sandwich_circuit(n, int(rng.integers(1, 30)), int(rng.integers(1 << 30)))
        elif mix < 0.85 and n >= 2:
            gl = W.tfim_gates(n, int(rng.integers(1, 30)), 0.05, 1.0, W.tfim_fields(n, 3), order=int(rng.integers(1, 3)))
        else:
            kinds = ["H", "RZZ", "CP", "RX", "SWAP", "CX"] if n > 1 else ["H", "RX"]
            gl = W.qft_gates(n) + W.random_circuit(n, 20, int(rng.integers(1 << 30)), kinds)
        psi0 = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
        out.append((f"trial {trial} n={n}", n, gl, cfg, psi0 / np.linalg.norm(psi0)))
    return out


@pytest.mark.parametrize("seed", [1, 4, 5])
def test_random_plans_build_and_match_oracle(tmp_path, qs, seed):
    if not plan_host.available():
        pytest.skip("needs g++ and the CUDA headers")
    cases = _cases(seed, 200)
    res = plan_host.interpret(qs, [c[:4] for c in cases], str(tmp_path), [c[4][None, :] for c in cases])
    bad = []
    for (name, n, gl, cfg, psi0), (got, _) in zip(cases, res):
        ref = oracle.simulate(n, gl, psi0)
        err = np.linalg.norm(got[0] - ref) / np.linalg.norm(ref)
        if not err <= (6e-2 if cfg[3] == 3 else 1e-4):
            bad.append((name, cfg, err))
    assert not bad, bad


def _batch_cases(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for trial in range(count):
        n, B = int(rng.integers(2, 11)), int(rng.integers(2, 4))
        cfg = (int(rng.choice([0, 3, 5, 7, 9, 12, 13])), int(rng.choice([0, 1, 2, 3, 4])),
               int(rng.choice([0, 1, 2, 3, 4, 5])), int(rng.choice([0, 0, 1, 2, 3])), int(rng.choice([0, 3, 4, 5])))
        gl, P = [], 0
        for _ in range(int(rng.integers(1, 60))):
            r = rng.random()
            if r < 0.45:
                gl.append(W.Gate(str(rng.choice(["RX", "RY", "RZ"])), (int(rng.integers(n)),), (0.0,), None, P))
                P += 1
            elif r < 0.7:
                a, b = (int(x) for x in rng.choice(n, 2, replace=False))
                gl.append(W.Gate(str(rng.choice(["RZZ", "CP"])), (a, b), (0.0,), None, P))
                P += 1
            else:
                k = str(rng.choice(["H", "CX", "SX", "CZ", "SWAP", "T"]))
                gl.append(W.Gate(k, tuple(int(x) for x in rng.choice(n, W.arity(k), replace=False))))
        if P == 0:
            gl.append(W.Gate("RX", (0,), (0.0,), None, 0))
            P = 1
        params = rng.uniform(-3, 3, size=(B, P))
        psi0 = rng.standard_normal((B, 2 ** n)) + 1j * rng.standard_normal((B, 2 ** n))
        out.append((f"batch trial {trial} n={n} B={B}", n, gl, cfg, params,
                    psi0 / np.linalg.norm(psi0, axis=1, keepdims=True)))
    return out


def test_random_batched_plans_match_oracle(tmp_path, qs):
    # one plan per parameter vector, merged into per-item constants when the
    # items' plans agree (as the executor runs them)
    if not plan_host.available():
        pytest.skip("needs g++ and the CUDA headers")
    cases = _batch_cases(3, 120)
    res = plan_host.interpret(qs, [c[:5] for c in cases], str(tmp_path), [c[5] for c in cases])
    bad, merged = [], 0
    for (name, n, gl, cfg, params, psi0), (got, cnt) in zip(cases, res):
        merged += cnt["merged"]
        ref = np.stack([oracle.simulate(n, gl, psi0[b], theta=params[b]) for b in range(len(params))])
        err = np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1))
        if not err <= (6e-2 if cfg[3] == 3 else 1e-4):
            bad.append((name, cfg, err))
    assert not bad, bad
    assert merged > 100, merged
