"""Pins for the oracle against what the paper and the mathematics fix (CPU only).

Each test ties the oracle to something other than itself: textbook gate
identities and matrix exponentials of generators, an independent brute-force
simulator, the DFT / numpy ifft, GHZ and Grover closed forms, exact
diagonalisation, the Trotter-error table printed in Sec. 6.4, and finite
differences.  The last group plants mistakes in the oracle's gate
definitions (on the CPU) and checks that the pins catch them.
"""
import os

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from oracle import brute
from oracle import gates as og
import workloads as W

X = og.pauli("X")
Y = og.pauli("Y")
Z = og.pauli("Z")
I2 = og.pauli("I")


# --------------------------------------------------------------------------
# gate definitions (Sec. 3.2.2 gate library, OpenQASM table)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [0.0, 0.3, -1.7, 2.9, 6.0])
def test_rotations_are_exponentials_of_generators(theta):
    m = og.matrix
    assert np.allclose(m("RX", (theta,)), expm(-0.5j * theta * X), atol=1e-14)
    assert np.allclose(m("RY", (theta,)), expm(-0.5j * theta * Y), atol=1e-14)
    assert np.allclose(m("RZ", (theta,)), expm(-0.5j * theta * Z), atol=1e-14)
    assert np.allclose(m("RZZ", (theta,)), expm(-0.5j * theta * np.kron(Z, Z)), atol=1e-14)
    assert np.allclose(m("RXX", (theta,)), expm(-0.5j * theta * np.kron(X, X)), atol=1e-14)
    assert np.allclose(m("RYY", (theta,)), expm(-0.5j * theta * np.kron(Y, Y)), atol=1e-14)
    P1 = np.diag([0, 1]).astype(complex)
    assert np.allclose(m("P", (theta,)), expm(1j * theta * P1), atol=1e-14)
    assert np.allclose(m("CP", (theta,)), expm(1j * theta * np.kron(P1, P1)), atol=1e-14)
    assert np.allclose(m("CRZ", (theta,)), expm(-0.5j * theta * np.kron(P1, Z)), atol=1e-14)
    assert np.allclose(m("CRX", (theta,)), expm(-0.5j * theta * np.kron(P1, X)), atol=1e-14)
    assert np.allclose(m("CRY", (theta,)), expm(-0.5j * theta * np.kron(P1, Y)), atol=1e-14)


def test_clifford_identities():
    m = og.matrix
    assert np.allclose(m("S") @ m("S"), Z)
    assert np.allclose(m("T") @ m("T"), m("S"))
    assert np.allclose(m("SX") @ m("SX"), X)
    assert np.allclose(m("SDG"), m("S").conj().T)
    assert np.allclose(m("TDG"), m("T").conj().T)
    assert np.allclose(m("H") @ Z @ m("H"), X)
    assert np.allclose(m("H") @ m("H"), I2)
    # V = S H satisfies V Z V^dagger = Y (Sec. 5.1 YY conjugation)
    V = m("S") @ m("H")
    assert np.allclose(V @ Z @ V.conj().T, Y)
    # U3 special cases (OpenQASM 2.0)
    th = 0.77
    assert np.allclose(m("U3", (th, -np.pi / 2, np.pi / 2)), m("RX", (th,)))
    assert np.allclose(m("U3", (th, 0.0, 0.0)), m("RY", (th,)))
    assert np.allclose(m("U2", (0.0, np.pi)), m("H"))
    assert np.allclose(m("ISWAP"), expm(0.25j * np.pi * (np.kron(X, X) + np.kron(Y, Y))))
    # permutation gates on basis states
    sw = m("SWAP")
    assert sw[1, 2] == 1 and sw[2, 1] == 1
    ccx = m("CCX")
    assert ccx[6, 7] == 1 and ccx[7, 6] == 1 and np.allclose(np.diag(ccx)[:6], 1)
    cs = m("CSWAP")
    assert cs[5, 6] == 1 and cs[6, 5] == 1 and np.allclose(np.diag(cs)[:5], 1)
    for k in W.ONE_QUBIT + W.TWO_QUBIT + W.THREE_QUBIT:
        if k == "U":
            continue
        U = m(k, tuple(0.4 + 0.3 * i for i in range(W.N_PARAMS.get(k, 0))))
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-14), k


# --------------------------------------------------------------------------
# the application loop vs two independent formulations
# --------------------------------------------------------------------------
def test_wire_order_bell_and_cx():
    # qubit 0 is the most significant bit (Sec. 3.2.2, App. A: "qubit q is bit n-1-q")
    psi = oracle.simulate(2, [W.Gate("X", (0,)), W.Gate("CX", (0, 1))])
    assert np.allclose(psi, [0, 0, 0, 1])
    psi = oracle.simulate(2, [W.Gate("X", (1,)), W.Gate("CX", (0, 1))])
    assert np.allclose(psi, [0, 1, 0, 0])
    # Bell state of Sec. 6.1: (H x I) CNOT |00> = (|00> + |11>)/sqrt 2
    psi = oracle.simulate(2, [W.Gate("H", (0,)), W.Gate("CX", (0, 1))])
    assert np.allclose(psi, np.array([1, 0, 0, 1]) / np.sqrt(2))


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (4, 4), (5, 5), (6, 6)])
def test_oracle_matches_brute_force(n, seed):
    gl = W.random_circuit(n, 60, seed)
    psi0 = W.random_state(n, seed + 100)
    a = oracle.simulate(n, gl, psi0)
    b = brute.einsum_apply(psi0, n, gl)
    c = brute.full_unitary(n, gl) @ psi0
    assert np.max(np.abs(a - b)) < 1e-12
    assert np.max(np.abs(a - c)) < 1e-12


def test_norm_preserved_n10():
    gl = W.random_circuit(10, 300, 7)
    psi = oracle.simulate(10, gl, W.random_state(10, 8))
    assert abs(np.linalg.norm(psi) - 1) < 1e-12


# --------------------------------------------------------------------------
# QFT, WHT, GHZ, Gray-code ladder, Grover
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 5, 8])
def test_qft_basis_state_is_dft_column(n):
    N = 1 << n
    gl = W.qft_gates(n, swaps=True)
    for j in [0, 1, 5 % N, N - 1]:
        psi0 = np.zeros(N, complex)
        psi0[j] = 1
        out = oracle.simulate(n, gl, psi0)
        k = np.arange(N)
        ref = np.exp(2j * np.pi * j * k / N) / np.sqrt(N)   # Sec. 3.2.3 QFT definition
        assert np.max(np.abs(out - ref)) < 1e-12


@pytest.mark.parametrize("n", [4, 7, 12])
def test_qft_is_sqrtN_ifft(n):
    psi0 = W.random_state(n, 11)
    out = oracle.simulate(n, W.qft_gates(n, swaps=True), psi0)
    ref = np.sqrt(1 << n) * np.fft.ifft(psi0)
    assert np.max(np.abs(out - ref)) < 1e-12
    # without the final swaps the result is the bit-reversed permutation
    out2 = oracle.simulate(n, W.qft_gates(n, swaps=False), psi0)
    rev = np.array([int(format(i, f"0{n}b")[::-1], 2) for i in range(1 << n)])
    assert np.max(np.abs(out2 - ref[rev])) < 1e-12


def test_qft_gate_counts_match_paper():
    # 25-qubit gate-stream QFT without swaps has 325 gates (Sec. 4.1); with swaps
    # at 12 qubits: 78 gates + 6 swaps
    assert len(W.qft_gates(25, swaps=False)) == 325
    assert len(W.qft_gates(12, swaps=True)) == 78 + 6
    assert len(W.qft_gates(30, swaps=True)) == 30 + 435 + 15


def test_wht_twice_identity_and_uniform():
    n = 9
    psi0 = W.random_state(n, 3)
    out = oracle.simulate(n, W.wht_gates(n) + W.wht_gates(n), psi0)
    assert np.max(np.abs(out - psi0)) < 1e-12
    u = oracle.simulate(n, W.wht_gates(n))
    assert np.allclose(u, np.full(1 << n, 2 ** (-n / 2)), atol=1e-14)
    # H^{x4} entries are (1/4)(-1)^{popcount(r & c)} (App. A)
    M = brute.full_unitary(4, W.wht_gates(4))
    r = np.arange(16)
    pc = np.array([[bin(a & b).count("1") for b in r] for a in r])
    assert np.allclose(M, 0.25 * (-1.0) ** pc, atol=1e-14)


@pytest.mark.parametrize("n", [2, 5, 11])
def test_ghz(n):
    psi = oracle.simulate(n, W.ghz_gates(n))
    ref = np.zeros(1 << n, complex)
    ref[0] = ref[-1] = 1 / np.sqrt(2)                      # Sec. 3.2.3 GHZ
    assert np.max(np.abs(psi - ref)) < 1e-14


@pytest.mark.parametrize("n", [3, 6, 10])
def test_ascending_cnot_ladder_is_gray_code_gather(n):
    psi0 = W.random_state(n, 21)
    out = oracle.simulate(n, W.cnot_ladder(n), psi0)
    y = np.arange(1 << n)
    assert np.array_equal(out, psi0[y ^ (y >> 1)])        # bit-exact permutation


@pytest.mark.parametrize("n,marked", [(2, [3]), (3, [5]), (3, [1, 6])])
def test_grover_success_probability(n, marked):
    N = 1 << n
    th = np.arcsin(np.sqrt(len(marked) / N))
    for k in range(0, 4):
        psi = oracle.simulate(n, W.grover_gates(n, marked, k))
        p = float(np.sum(np.abs(psi[marked]) ** 2))
        assert abs(p - np.sin((2 * k + 1) * th) ** 2) < 1e-12


# --------------------------------------------------------------------------
# TFIM: the printed Trotter table (Sec. 6.4) and exact diagonalisation
# --------------------------------------------------------------------------
def _golden_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "trotter_error_n6.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            r, l2, mae, inf = line.split()
            rows.append((int(r), float(l2), float(mae), float(inf)))
    return rows


def _exact_tfim(n, J, h, t):
    H = brute.pauli_sum_matrix(n, W.tfim_paulis(n, J, h))
    psi0 = np.zeros(1 << n, complex)
    psi0[0] = 1
    return expm(-1j * H * t) @ psi0


def test_first_order_trotter_table_reproduced():
    n, J, h, t = 6, 1.0, 0.5, 1.0
    ex = _exact_tfim(n, J, h, t)
    for (r, l2, mae, inf) in _golden_rows():
        psi = oracle.simulate(n, W.tfim_gates(n, r, t / r, J, h, order=1))
        got_l2 = np.linalg.norm(psi - ex)
        got_mae = np.mean(np.abs(np.abs(psi) ** 2 - np.abs(ex) ** 2))
        got_inf = 1 - abs(np.vdot(ex, psi)) ** 2
        for got, printed in ((got_l2, l2), (got_mae, mae), (got_inf, inf)):
            # printed with 3 significant digits: agree to half a unit in the last digit
            ulp = 10 ** (np.floor(np.log10(printed)) - 2)
            assert abs(got - printed) <= 0.5 * ulp + 1e-15, (r, got, printed)


def test_second_order_trotter_error_scaling():
    n, J, t = 6, 1.0, 1.0
    h = W.tfim_fields(n, 3)
    H = brute.pauli_sum_matrix(n, [(-J, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
                               + [(float(h[i]), 1 << i, 0) for i in range(n)])
    psi0 = np.zeros(1 << n, complex)
    psi0[0] = 1
    ex = expm(-1j * H * t) @ psi0
    errs = []
    for r in (8, 16, 32):
        psi = oracle.simulate(n, W.tfim_gates(n, r, t / r, J, h, order=2))
        errs.append(np.linalg.norm(psi - ex))
    # second order: amplitude error falls ~4x per halving of dt
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.5 < errs[1] / errs[2] < 4.5


# --------------------------------------------------------------------------
# expectations and gradients
# --------------------------------------------------------------------------
def test_expectation_matches_dense_hamiltonian():
    n = 6
    rng = np.random.default_rng(5)
    terms = [(float(rng.normal()), int(rng.integers(64)), int(rng.integers(64))) for _ in range(12)]
    terms += W.tfim_paulis(n, 1.0, 1.0)
    # Hermitian: each Pauli string is Hermitian, real coefficients
    psi = W.random_state(n, 9)
    H = brute.pauli_sum_matrix(n, terms)
    assert abs(oracle.expect(psi, n, terms) - np.vdot(psi, H @ psi).real) < 1e-12
    # basis states and |+>^n
    b = np.zeros(64, complex)
    b[0b101100] = 1
    assert oracle.expect(b, n, [(1.0, 0, 1 << 0)]) == pytest.approx(-1.0)   # qubit 0 = MSB = 1
    assert oracle.expect(b, n, [(1.0, 0, 1 << 1)]) == pytest.approx(1.0)
    plus = np.full(64, 1 / 8, complex)
    for q in range(n):
        assert oracle.expect(plus, n, [(1.0, 1 << q, 0)]) == pytest.approx(1.0)


def test_param_shift_matches_finite_differences_and_analytic():
    n, L = 4, 2
    gl = W.vqe_ansatz_gates(n, L)
    theta = W.vqe_params(n, L, 1, 6)[0]
    terms = W.tfim_paulis(n, 1.0, 1.0)
    ps = oracle.param_shift_grad(n, gl, theta, terms)
    fd = oracle.finite_diff_grad(n, gl, theta, terms, eps=1e-5)
    assert np.max(np.abs(ps - fd)) < 1e-8
    # analytic derivative of one parameter through the brute-force unitary
    H = brute.pauli_sum_matrix(n, terms)
    psi0 = np.zeros(1 << n, complex)
    psi0[0] = 1
    i = 5
    eps = 1e-6
    tp, tm = theta.copy(), theta.copy()
    tp[i] += eps
    tm[i] -= eps
    ep = np.vdot(brute.full_unitary(n, gl, tp) @ psi0, H @ (brute.full_unitary(n, gl, tp) @ psi0)).real
    em = np.vdot(brute.full_unitary(n, gl, tm) @ psi0, H @ (brute.full_unitary(n, gl, tm) @ psi0)).real
    assert abs(ps[i] - (ep - em) / (2 * eps)) < 1e-7


def test_maxcut_expectation_two_routes():
    rng = np.random.default_rng(1)
    n = 8
    edges = W.random_regular3_graph(n, rng)
    assert all(d == 3 for d in np.bincount(np.array(edges).ravel(), minlength=n))
    gam, bet = [0.7, 0.2], [0.3, 1.1]
    psi = oracle.simulate(n, W.qaoa_gates(n, edges, gam, bet))
    c1 = oracle.expected_cut(psi, n, edges)
    c2 = oracle.expect(psi, n, W.maxcut_paulis(n, edges))
    assert abs(c1 - c2) < 1e-12
    assert 0 <= c1 <= len(edges)


def test_qaoa_single_edge_closed_form():
    # one edge, p = 1: <C> = 1/2 + (1/2) sin(4 beta) sin(gamma) for
    # e^{-i beta (X1+X2)} e^{-i gamma (1 - Z1 Z2)/2} |++>
    for gam, bet in [(0.3, 0.2), (1.1, 0.7), (2.5, 1.3)]:
        psi = oracle.simulate(2, W.qaoa_gates(2, [(0, 1)], [gam], [bet]))
        c = oracle.expected_cut(psi, 2, [(0, 1)])
        assert abs(c - (0.5 + 0.5 * np.sin(4 * bet) * np.sin(gam))) < 1e-12


# --------------------------------------------------------------------------
# planted mistakes (in the oracle, on the CPU) must be caught by the pins
# --------------------------------------------------------------------------
def _mutated(monkeypatch, kind, fn):
    orig = og.matrix

    def m(k, params=(), mat=None):
        U = orig(k, params, mat)
        return fn(U) if k == kind else U
    monkeypatch.setattr(og, "matrix", m)


def test_planted_cphase_sign_error_is_caught(monkeypatch):
    _mutated(monkeypatch, "CP", lambda U: U.conj())
    n = 5
    psi0 = W.random_state(n, 11)
    out = oracle.simulate(n, W.qft_gates(n), psi0)
    assert np.max(np.abs(out - np.sqrt(32) * np.fft.ifft(psi0))) > 1e-3


def test_planted_transposed_cx_is_caught(monkeypatch):
    # a transposed (control/target swapped) CNOT breaks the Gray-code pin
    _mutated(monkeypatch, "CX", lambda U: U[[0, 3, 2, 1]][:, [0, 3, 2, 1]])
    n = 6
    psi0 = W.random_state(n, 21)
    out = oracle.simulate(n, W.cnot_ladder(n), psi0)
    y = np.arange(1 << n)
    assert not np.array_equal(out, psi0[y ^ (y >> 1)])


def test_planted_rx_half_angle_error_is_caught(monkeypatch):
    _mutated(monkeypatch, "RX", lambda U: U @ U)
    n, J, h, t = 6, 1.0, 0.5, 1.0
    ex = _exact_tfim(n, J, h, t)
    psi = oracle.simulate(n, W.tfim_gates(n, 4, t / 4, J, h, order=1))
    assert abs((1 - abs(np.vdot(ex, psi)) ** 2) - 4.88e-2) > 1e-3
