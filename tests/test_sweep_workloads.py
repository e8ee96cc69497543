"""The end-to-end sweep's workloads (the paper's gate-based suite: TFIM,
long-range Ising, Heisenberg chain / XXZ / random field / 2-leg ladder,
variational ansatze, QCBM, GHZ, graph state, QFT, phase estimation, QAOA
ring, Deutsch-Jozsa, random circuit, amplitude estimation, W state, Grover
search with a CCX V-chain, coined quantum walk).

1. The generators are pinned by what their circuits must do, evaluated with
   the oracle: W-state amplitudes, phase estimation of a dyadic phase landing
   on one index, a balanced Deutsch-Jozsa oracle never returning the zero
   input, Grover's sin^2((2k+1) theta) with clean ancillas, the quantum walk
   against the classical amplitude recursion, graph-state stabilisers, magnetisation conservation of the
   bond-by-bond Heisenberg ladder, the first-order error law of the
   layer-ordered Heisenberg chains against exact evolution, and the
   long-range Ising phases from their closed form.
2. Every family's fused plan, under several tile shapes, is interpreted on the
   host pass by pass and matches the oracle (relative L2 <= 1e-4)."""
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


def _weights(n):
    return np.array([bin(x).count("1") for x in range(2 ** n)])


def test_w_state_amplitudes():
    for n in (3, 5, 8):
        psi = oracle.simulate(n, W.w_state_gates(n))
        w = _weights(n)
        assert np.allclose(np.abs(psi[w == 1]), 1 / np.sqrt(n), atol=1e-12)
        assert np.max(np.abs(psi[w != 1])) < 1e-12


def test_exact_phase_estimation_lands_on_one_index():
    for n, seed in ((6, 1), (9, 2)):
        m = n - 1
        phi = W.qpe_exact_phase(n, seed)
        j = int(round(phi / (2 * np.pi) * 2 ** m))
        p = np.abs(oracle.simulate(n, W.qpe_gates(n, phi))) ** 2
        # counting qubits 0..m-1 hold j (qubit 0 most significant), the target stays |1>
        assert p[(j << 1) | 1] > 1 - 1e-12
    # the inexact phase spreads over several indices
    p = np.abs(oracle.simulate(7, W.qpe_gates(7, 0.4))) ** 2
    assert np.max(p) < 0.99 and abs(p.sum() - 1) < 1e-12


def test_grover_vchain_success_probability():
    # sin^2((2k+1) theta), sin theta = 2^(-m/2), on m data qubits; the V-chain ancillas end in |0>
    for n, marked, k in ((5, 2, 1), (9, 37, 3), (10, 5, 2)):
        m = (n + 3) // 2
        p = np.abs(oracle.simulate(n, W.grover_vchain_gates(n, marked, k))) ** 2
        th = np.arcsin(2.0 ** (-m / 2))
        assert abs(p[marked << (n - m)] - np.sin((2 * k + 1) * th) ** 2) < 1e-12
        assert abs(p.reshape(2 ** m, -1)[:, 0].sum() - 1) < 1e-12


def test_quantum_walk_matches_classical_recursion():
    # amplitudes psi(c, x) of the coined walk on the 2^p cycle, step: coin H, x +- 1
    for n, steps in ((6, 5), (9, 4)):
        p = n // 2
        amp = np.zeros((2, 2 ** p), complex)
        amp[:, 0] = np.array([1, 1j]) / np.sqrt(2)
        for _ in range(steps):
            h0, h1 = (amp[0] + amp[1]) / np.sqrt(2), (amp[0] - amp[1]) / np.sqrt(2)
            amp = np.stack([np.roll(h0, -1), np.roll(h1, 1)])
        psi0 = np.zeros(2 ** n, complex)
        psi0[0], psi0[1 << (n - 1)] = 1 / np.sqrt(2), 1j / np.sqrt(2)
        psi = oracle.simulate(n, W.quantum_walk_gates(n, steps), psi0)
        want = np.zeros(2 ** n, complex)
        for c in range(2):
            for x in range(2 ** p):
                idx = c << (n - 1)
                for j in range(p):
                    idx |= ((x >> j) & 1) << (n - 2 - j)   # position bit j = qubit 1 + j
                want[idx] = amp[c, x]
        assert np.max(np.abs(psi - want)) < 1e-12


def test_deutsch_jozsa_balanced_oracle():
    for n, seed in ((5, 3), (8, 4)):
        p = np.abs(oracle.simulate(n, W.deutsch_jozsa_gates(n, seed))) ** 2
        # inputs are qubits 0..n-2 (index bits n-1..1): all-zero input means index 0 or 1
        assert p[0] + p[1] < 1e-12


def test_graph_state_stabilisers():
    n = 7
    gl = W.graph_state_gates(n, 5, chords=3)
    psi = oracle.simulate(n, gl)
    edges = [g.wires for g in gl if g.kind == "CZ"]
    for v in range(n):
        z = 0
        for a, b in edges:
            if v in (a, b):
                z |= 1 << (b if a == v else a)
        assert abs(oracle.expect(psi, n, [(1.0, 1 << v, z)]) - 1) < 1e-12


def test_heisenberg_ladder_conserves_magnetisation():
    # each bond's XX . YY . ZZ product commutes with the total Z
    n = 8
    psi0 = np.zeros(2 ** n, complex)
    psi0[0b10110010] = 1.0
    psi = oracle.simulate(n, W.heisenberg_ladder_gates(n, 3, 0.1), psi0)
    w = _weights(n)
    assert np.max(np.abs(psi[w != 4])) < 1e-12
    assert np.max(np.abs(psi[w == 4])) < 1 - 1e-3   # the state did move


@pytest.mark.parametrize("delta,fields", [(1.0, None), (0.5, None), (1.0, "random")])
def test_heisenberg_chain_is_a_first_order_product_formula(delta, fields):
    # one step against exp(-i H dt), H = J sum (XX + YY + delta ZZ) + sum h_i Z_i:
    # the local error of a first-order product formula falls 4x per halving of dt
    from scipy.linalg import expm
    from oracle import brute
    n, J = 6, 0.9
    h = np.linspace(-1, 1, n) if fields else None
    terms = []
    for b in range(n - 1):
        m = (1 << b) | (1 << (b + 1))
        terms += [(J, m, 0), (J, m, m), (J * delta, 0, m)]
    if h is not None:
        terms += [(float(h[q]), 0, 1 << q) for q in range(n)]
    H = brute.pauli_sum_matrix(n, terms)
    psi0 = W.random_state(n, 3)
    errs = []
    for dt in (0.04, 0.02):
        got = oracle.simulate(n, W.heisenberg_gates(n, 1, dt, J=J, delta=delta, fields=h), psi0)
        errs.append(np.linalg.norm(got - expm(-1j * H * dt) @ psi0))
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_long_range_ising_phases():
    n, dt, J, alpha = 6, 0.07, 1.3, 1.5
    gl = W.long_range_ising_gates(n, 1, dt, J=J, h=0.0, alpha=alpha)
    for x in (0, 5, 37, 63):
        psi0 = np.zeros(2 ** n, complex)
        psi0[x] = 1
        got = oracle.simulate(n, gl, psi0)[x]
        z = [1 - 2 * ((x >> (n - 1 - q)) & 1) for q in range(n)]
        ph = sum(J * dt / (j - i) ** alpha * z[i] * z[j] for i in range(n) for j in range(i + 1, n))
        assert abs(got - np.exp(1j * ph)) < 1e-12


def test_sweep_plans_interpreted_on_host_match_oracle(tmp_path, qs):
    if not plan_host.available():
        pytest.skip("needs g++ and the CUDA headers")
    n = 12
    cases, psi0s, expect = [], [], []
    shapes = [(0, 0, 0, 0, 0), (10, 4, 4, 0, 0), (9, 3, 5, 0, 0)]
    for k, (name, gl) in enumerate(W.sweep_workloads(n)):
        sh = shapes[k % len(shapes)]
        cases.append((name, n, gl, sh))
        rng = np.random.default_rng(50 + k)
        psi0 = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
        psi0 /= np.linalg.norm(psi0)
        psi0s.append(psi0[None, :])
        expect.append(oracle.simulate(n, gl, psi0))
    res = plan_host.interpret(qs, cases, str(tmp_path), psi0s)
    bad = []
    for (name, _, _, sh), (got, _), ref in zip(cases, res, expect):
        err = np.linalg.norm(got[0] - ref) / np.linalg.norm(ref)
        if not err < 1e-4:
            bad.append((name, sh, err))
    assert not bad, bad
