"""Adjoint gradients (qs_grad, a layer at a time) against the oracle.

The oracle's parameter shift, [E(t + pi/2) - E(t - pi/2)] / 2, is exact for
gates exp(-i t G / 2) with G^2 = I (and for CP, whose generator has
eigenvalues 0 and 1); the oracle's central finite difference (complex128,
eps = 1e-5) is a second, independent check.  Tolerance 2e-5 per component:
the adjoint sums FP32 products of two complex64 states in FP64, and
|dE/dt| <= sum |coeff| for these Hamiltonians.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_19147_gb300 as qs  # noqa: E402


def _grad(n, gl, theta, terms):
    st = qs.State(n, batch=theta.shape[0])
    e, g = st.grad(gl, theta, terms)
    st.close()
    return e, g


def test_generators_transported_through_later_gates_of_the_layer():
    # one long 1q run per wire with fixed gates between the rotations: the
    # gradient of an early rotation needs V G V^dagger, V = the later gates
    n = 5
    gl, k = [], 0
    for q in range(n):
        gl += [W.Gate("RX", (q,), (0.0,), None, k), W.Gate("H", (q,)), W.Gate("RY", (q,), (0.0,), None, k + 1),
               W.Gate("S", (q,)), W.Gate("RZ", (q,), (0.0,), None, k + 2), W.Gate("T", (q,)),
               W.Gate("RX", (q,), (0.0,), None, k + 3)]
        k += 4
    gl += [W.Gate("CX", (q, q + 1)) for q in range(n - 1)]
    gl += [W.Gate("RY", (q,), (0.0,), None, k + q) for q in range(n)]
    P = k + n
    theta = np.random.default_rng(11).uniform(0, 2 * np.pi, size=(2, P))
    terms = W.tfim_paulis(n, 1.0, 0.7) + [(0.3, 0b00110, 0b00011), (-0.2, 0b10001, 0)]
    e, g = _grad(n, gl, theta, terms)
    for b in range(2):
        assert abs(e[b] - oracle.energy(n, gl, theta[b], terms)) < 1e-5
        ps = oracle.param_shift_grad(n, gl, theta[b], terms)
        assert np.max(np.abs(g[b] - ps)) < 2e-5, np.max(np.abs(g[b] - ps))


def test_mixed_layers_every_inverse_kind():
    # rotations between multi-qubit gates of every inverse rule (self-inverse,
    # negated angle, ISWAP), parameterised RZZ / CP, a parameter shared by two
    # gates (contributions add; checked by finite differences)
    n = 6
    gl = [W.Gate("H", (q,)) for q in range(n)]
    gl += [W.Gate("RY", (q,), (0.0,), None, q) for q in range(n)]
    gl += [W.Gate("ISWAP", (0, 1)), W.Gate("CRX", (2, 3), (0.7,)), W.Gate("CCX", (1, 4, 5)),
           W.Gate("RZZ", (2, 5), (0.0,), None, n), W.Gate("SWAP", (0, 4)), W.Gate("CP", (1, 3), (0.0,), None, n + 1),
           W.Gate("RXX", (0, 5), (0.4,)), W.Gate("CSWAP", (3, 0, 2)), W.Gate("CH", (4, 1))]
    gl += [W.Gate("RZ", (q,), (0.0,), None, n + 2 + q) for q in range(n)]
    gl += [W.Gate("U3", (2,), (0.3, 0.8, -0.4)), W.Gate("RX", (2,), (0.0,), None, 2)]   # shared index 2
    P = 2 * n + 2
    theta = np.random.default_rng(12).uniform(0, 2 * np.pi, size=(3, P))
    terms = W.tfim_paulis(n, 0.8, 1.1) + [(0.25, 0b101000, 0b001001)]
    e, g = _grad(n, gl, theta, terms)
    for b in range(3):
        assert abs(e[b] - oracle.energy(n, gl, theta[b], terms)) < 1e-5
        fd = oracle.finite_diff_grad(n, gl, theta[b], terms)
        assert np.max(np.abs(g[b] - fd)) < 2e-5, np.max(np.abs(g[b] - fd))


def test_vqe_ansatz_n10_against_param_shift_and_fd():
    # the adjoint config's ansatz and Hamiltonian at n = 10 (full check)
    n, L, B = 10, 4, 2
    gl = W.vqe_ansatz_gates(n, L)
    theta = W.vqe_params(n, L, B, 6)
    terms = W.tfim_paulis(n, 1.0, 1.0)
    e, g = _grad(n, gl, theta, terms)
    for b in range(B):
        ps = oracle.param_shift_grad(n, gl, theta[b], terms)
        assert np.max(np.abs(g[b] - ps)) < 2e-5
    fd = oracle.finite_diff_grad(n, gl, theta[0], terms, indices=range(0, 2 * n * L, 7))
    assert np.max(np.abs(g[0][::7] - fd)) < 2e-5


def test_vqe_config_full_size_sampled():
    # n = 24, 12 layers, 576 parameters, batch 32: energies of all items
    # against qs_expect on the forward states, and oracle parameter shift on
    # two sampled parameters of one item (energy within the oracle tolerance)
    n, L, B = 24, 12, 32
    gl = W.vqe_ansatz_gates(n, L)
    theta = W.vqe_params(n, L, B, 6)
    terms = W.tfim_paulis(n, 1.0, 1.0)
    st = qs.State(n, batch=B)
    e, g = st.grad(gl, theta, terms)
    e2 = st.expect(terms)
    st.close()
    assert np.all(np.isfinite(g)) and g.shape == (B, 2 * n * L)
    # qs_grad takes E = Re <psi|H psi> from the FP32 lam = H psi; qs_expect sums
    # the Pauli terms directly: the two differ by FP32 rounding only
    assert np.max(np.abs(e - e2)) < 1e-5
    assert np.max(np.abs(g)) <= sum(abs(t[0]) for t in terms)
    idx = [5, 2 * n * L - 2]
    ps = oracle.param_shift_grad(n, gl, theta[3], terms, indices=idx)
    assert np.max(np.abs(g[3][idx] - ps)) < 2e-5, (g[3][idx], ps)


def test_autograd_function_against_param_shift_fd_and_chain_rule():
    # qs_expectation (the torch.autograd.Function over qs_grad) driven through
    # torch.autograd.grad at n = 10: energies against the oracle, gradients
    # against oracle parameter shift and finite differences, and the chain rule
    # with a non-unit upstream gradient; results stay on the CUDA device
    n, L, B = 10, 3, 3
    gl = W.vqe_ansatz_gates(n, L)
    theta = W.vqe_params(n, L, B, 17)
    terms = W.tfim_paulis(n, 1.0, 1.0)
    p = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    e = qs.qs_expectation(p, n, gl, terms)
    assert e.is_cuda and e.shape == (B,)
    w = torch.tensor([0.5, -2.0, 3.0], dtype=torch.float64, device="cuda")
    (gp,) = torch.autograd.grad((w * e).sum(), p)
    assert gp.is_cuda and gp.shape == p.shape
    gp = gp.cpu().numpy()
    for b in range(B):
        assert abs(e[b].item() - oracle.energy(n, gl, theta[b], terms)) < 1e-5
        ps = oracle.param_shift_grad(n, gl, theta[b], terms)
        assert np.max(np.abs(gp[b] - w[b].item() * ps)) < 2e-5 * abs(w[b].item())
    fd = oracle.finite_diff_grad(n, gl, theta[1], terms, indices=range(0, 2 * n * L, 5))
    assert np.max(np.abs(gp[1][::5] / w[1].item() - fd)) < 2e-5
    # a second call reuses the cached state and gives the same energies
    e2 = qs.qs_expectation(p.detach(), n, gl, terms)
    assert torch.allclose(e2, e.detach(), rtol=0, atol=1e-12)
