"""GPU parity: the CUDA path (through the C ABI) against the complex128 oracle.

Tolerances (from the stated target and the paper's parity budgets, Sec. 5.3
and Sec. 6.2): max |d amplitude| <= 2e-5, fidelity >= 1 - 1e-6, relative L2
<= 1e-5 (<= 1e-4 for the 100-step TFIM run, where ~10^4 complex64 roundings
accumulate); permutation layers bit-exact.
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


def _metrics(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    d = np.max(np.abs(got - ref))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    return d, rel, fid


def _run(n, gates, psi0=None, mode="fused", **kw):
    st = qs.State(n)
    if psi0 is not None:
        st.set(psi0.astype(np.complex64))
    st.apply(gates, mode=mode, **kw)
    out = st.get()[0]
    st.close()
    return out


def _ref(n, gates, psi0=None):
    p = None if psi0 is None else psi0.astype(np.complex64).astype(np.complex128)
    return oracle.simulate(n, gates, p)


def _assert_close(got, ref, tol_rel=1e-5):
    d, rel, fid = _metrics(got, ref)
    assert d <= 2e-5, d
    assert rel <= tol_rel, rel
    assert fid >= 1 - 1e-6, fid


@pytest.mark.parametrize("mode", ["fused", "pergate"])
def test_qft12_random_state(mode):
    n = 12
    psi0 = W.random_state(n, 1)
    gl = W.qft_gates(n, swaps=True)
    _assert_close(_run(n, gl, psi0, mode), _ref(n, gl, psi0))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 9, 12, 13, 14, 17])
@pytest.mark.parametrize("mode", ["fused", "pergate"])
def test_random_circuits_all_kinds(n, mode):
    gl = W.random_circuit(n, 150, 1000 + n)
    psi0 = W.random_state(n, 2000 + n)
    _assert_close(_run(n, gl, psi0, mode), _ref(n, gl, psi0))


@pytest.mark.parametrize("tq,lq", [(13, 4), (12, 5), (10, 3), (8, 2), (13, 6)])
def test_tile_shapes(tq, lq):
    n = 18
    gl = W.random_circuit(n, 200, 77, kinds=["H", "RX", "U", "CX", "CZ", "RZZ", "SWAP", "CP", "RY", "CCX"])
    psi0 = W.random_state(n, 78)
    _assert_close(_run(n, gl, psi0, tile_qubits=tq, low_qubits=lq), _ref(n, gl, psi0))


@pytest.mark.parametrize("n", [16, 20])
def test_haar_layers(n):
    gl = []
    rng = np.random.default_rng(5)
    for _ in range(3):
        gl += [W.Gate("U", (q,), (), W.haar_u2(rng)) for q in range(n)]
    psi0 = W.random_state(n, 6)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))


def _u2_of(c, s, rng):
    """diag(e^{ia}, e^{ib}) [[c, -s], [s, c]] diag(1, e^{id}) with random phases."""
    a, b, d = rng.uniform(0.0, 2.0 * np.pi, 3)
    return np.diag(np.exp(1j * np.array([a, b]))) @ np.array([[c, -s], [s, c]]) @ np.diag([1.0, np.exp(1j * d)])


def _u2_branch_matrix(kind, rng):
    # every branch of the phases-rotation-phases factorisation: Haar, diagonal
    # (s = 0), anti-diagonal (c = 0), |c| > |s|, |s| > |c|, |c| = |s|
    if kind == 0:
        return W.haar_u2(rng)
    th = {1: 0.0, 2: np.pi / 2, 3: 0.3, 4: 1.2, 5: np.pi / 4}[kind]
    return _u2_of(np.cos(th), np.sin(th), rng)


@pytest.mark.parametrize("tq,lq,gq", [(0, 0, 0), (13, 4, 0), (12, 5, 0), (13, 6, 0), (10, 3, 0),
                                      (13, 4, 4), (12, 4, 4), (13, 5, 4)])
def test_u2_layers_every_factorisation_branch(tq, lq, gq):
    # U(2) layers (split by CZ ladders so that they do not fuse) whose matrices
    # rotate through the branches, so that every group bit, the 16-byte pair
    # bit included, meets each rotation form
    n = 19
    rng = np.random.default_rng(11)
    gl = []
    for layer in range(7):
        gl += [W.Gate("U", (q,), (), _u2_branch_matrix((q + layer) % 6, rng)) for q in range(n)]
        gl += [W.Gate("CZ", (q, q + 1)) for q in range(n - 1)]
    # a scaled (non-unitary) layer keeps the general 2x2 path
    gl += [W.Gate("U", (q,), (), 0.97 * W.haar_u2(rng)) for q in range(n)]
    psi0 = W.random_state(n, 12)
    _assert_close(_run(n, gl, psi0, tile_qubits=tq, low_qubits=lq, group_qubits=gq), _ref(n, gl, psi0))


@pytest.mark.parametrize("tq,lq,gq", [(13, 4, 5), (13, 4, 4), (12, 4, 4), (12, 5, 5)])
def test_rotation_programs_every_group_size_against_oracle(tq, lq, gq):
    # Trotter steps whose rotation layers run as the specialised programs
    # (padded identities skipped, count-table diagonal between two layers),
    # at 4- and 5-bit register groups, against the oracle
    n = 20
    gl = W.tfim_gates(n, 6, 0.07, 1.0, W.tfim_fields(n, 13), order=2)
    psi0 = W.random_state(n, 14)
    _assert_close(_run(n, gl, psi0, tile_qubits=tq, low_qubits=lq, group_qubits=gq), _ref(n, gl, psi0))


@pytest.mark.parametrize("n", [10, 19, 21])
def test_qft_random_state(n):
    psi0 = W.random_state(n, 40 + n)
    gl = W.qft_gates(n, swaps=True)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))
    gl2 = W.qft_gates(n, swaps=False)
    _assert_close(_run(n, gl2, psi0), _ref(n, gl2, psi0))


@pytest.mark.parametrize("n", [6, 15, 22])
def test_permutation_layers_bit_exact(n):
    psi0 = W.random_state(n, 9).astype(np.complex64)
    y = np.arange(1 << n)
    # ascending CNOT ladder: out[y] = in[y ^ (y >> 1)], exact copy of amplitudes
    got = _run(n, W.cnot_ladder(n), psi0)
    assert np.array_equal(got, psi0[y ^ (y >> 1)])
    # SWAP / X run (bit permutation + xor): compare with the oracle on the widened input
    rng = np.random.default_rng(n)
    gl = []
    for _ in range(3 * n):
        a, b = rng.choice(n, 2, replace=False)
        gl.append(W.Gate("SWAP", (int(a), int(b))))
        gl.append(W.Gate("X", (int(rng.integers(n)),)))
    ref = oracle.simulate(n, gl, psi0.astype(np.complex128)).astype(np.complex64)
    assert np.array_equal(_run(n, gl, psi0), ref)
    # mixed X / CNOT / SWAP run through the general gather
    gl = []
    for _ in range(2 * n):
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        gl.append(W.Gate("CX", (a, b)))
        gl.append(W.Gate("X", (b,)))
    ref = oracle.simulate(n, gl, psi0.astype(np.complex128)).astype(np.complex64)
    assert np.array_equal(_run(n, gl, psi0), ref)
    assert np.array_equal(_run(n, gl, psi0, mode="pergate"), ref)


def test_ghz_and_wht():
    n = 20
    got = _run(n, W.ghz_gates(n))
    assert abs(got[0] - 2 ** -0.5) < 1e-7 and abs(got[-1] - 2 ** -0.5) < 1e-7
    assert np.count_nonzero(got) == 2
    psi0 = W.random_state(n, 3)
    _assert_close(_run(n, W.wht_gates(n) + W.wht_gates(n), psi0), psi0.astype(np.complex64).astype(complex))


@pytest.mark.parametrize("n", [12, 20])
def test_random_zz_and_long_range_diagonals(n):
    rng = np.random.default_rng(n)
    gl = [W.Gate("RZZ", (b, b + 1), (float(rng.uniform(0, 2 * np.pi)),)) for b in range(n - 1)]
    # all-distinct-angle all-to-all layer (Sec. 6.2 worst case)
    gl += [W.Gate("RZZ", (i, j), (float(rng.uniform(0, 2 * np.pi)),)) for i in range(n) for j in range(i + 1, n)]
    gl += [W.Gate("CP", (i, j), (float(rng.uniform(0, 2 * np.pi)),)) for i in range(0, n, 3) for j in range(1, n, 4) if i != j]
    gl += [W.Gate(k, (int(q),), (float(rng.uniform(0, 6)),) if k in ("RZ", "P") else ())
           for k, q in zip(["RZ", "P", "S", "T", "Z", "SDG"] * 3, rng.integers(0, n, 18))]
    psi0 = W.random_state(n, 8)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))


def test_suite_layers_n18():
    n = 18
    gl = W.suite28_gates(n, 3, 2, tail=True)
    psi0 = W.random_state(n, 12)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))


def test_tfim_second_order_n20():
    # config-3 parity size: 100 Strang steps, dt = 0.05, h_i ~ U[0.5, 1.5] (seed 3)
    n = 20
    gl = W.tfim_gates(n, 100, 0.05, 1.0, W.tfim_fields(n, 3), order=2)
    ref = _ref(n, gl)
    for mode in ("fused", "pergate"):
        got = _run(n, gl, mode=mode)
        d, rel, fid = _metrics(got, ref)
        assert d <= 2e-5 and rel <= 1e-4 and fid >= 1 - 1e-6, (mode, d, rel, fid)


def test_heisenberg_ladder_order_preserved():
    n = 10
    gl = []
    rng = np.random.default_rng(3)
    for _ in range(3):
        for b in range(n - 1):
            t = float(rng.uniform(0, 1))
            gl += [W.Gate("RXX", (b, b + 1), (t,)), W.Gate("RYY", (b, b + 1), (t,)), W.Gate("RZZ", (b, b + 1), (t,))]
    psi0 = W.random_state(n, 4)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))


def test_small_angle_not_dropped():
    n = 4
    psi0 = W.random_state(n, 5)
    gl = [W.Gate("RZ", (1,), (1e-6,)), W.Gate("H", (2,)), W.Gate("RZ", (2,), (1e-6,)), W.Gate("H", (2,))]
    got = _run(n, gl, psi0)
    ref = _ref(n, gl, psi0)
    _assert_close(got, ref)


def test_batched_states_and_params():
    n, L, B = 8, 2, 3
    gl = W.vqe_ansatz_gates(n, L)
    theta = W.vqe_params(n, L, B, 6)
    st = qs.State(n, batch=B)
    st.apply(gl, params=theta)
    got = st.get()
    st.close()
    for b in range(B):
        _assert_close(got[b], oracle.simulate(n, gl, theta=theta[b]))


def test_expectation_values():
    n, B = 14, 2
    psis = [W.random_state(n, 30 + b) for b in range(B)]
    st = qs.State(n, batch=B)
    st.set(np.stack(psis).astype(np.complex64))
    rng = np.random.default_rng(4)
    terms = W.tfim_paulis(n, 1.0, 0.7) + [(float(rng.normal()), int(rng.integers(1 << n)), int(rng.integers(1 << n)))
                                          for _ in range(20)]
    got = st.expect(terms)
    st.close()
    for b in range(B):
        ref = oracle.expect(psis[b].astype(np.complex64).astype(complex), n, terms)
        assert abs(got[b] - ref) < 1e-5 * max(1.0, sum(abs(t[0]) for t in terms)) / 10


def test_adjoint_gradient_matches_parameter_shift():
    n, L, B = 6, 2, 2
    gl = W.vqe_ansatz_gates(n, L)
    theta = W.vqe_params(n, L, B, 6)
    terms = W.tfim_paulis(n, 1.0, 1.0)
    st = qs.State(n, batch=B)
    e, g = st.grad(gl, theta, terms)
    st.close()
    for b in range(B):
        assert abs(e[b] - oracle.energy(n, gl, theta[b], terms)) < 1e-5
        ps = oracle.param_shift_grad(n, gl, theta[b], terms)
        assert np.max(np.abs(g[b] - ps)) < 2e-5, np.max(np.abs(g[b] - ps))


def test_adjoint_gradient_rzz_and_cp():
    n = 5
    gl = [W.Gate("H", (q,)) for q in range(n)]
    gl += [W.Gate("RZZ", (q, q + 1), (0.0,), None, q) for q in range(n - 1)]
    gl += [W.Gate("CP", (0, 3), (0.0,), None, n - 1), W.Gate("RX", (2,), (0.0,), None, n)]
    theta = np.random.default_rng(1).uniform(0, 2 * np.pi, size=(1, n + 1))
    terms = W.tfim_paulis(n, 1.0, 0.6) + [(0.4, 0b10010, 0b00110)]
    st = qs.State(n)
    e, g = st.grad(gl, theta, terms)
    st.close()
    ps = oracle.param_shift_grad(n, gl, theta[0], terms)
    assert np.max(np.abs(g[0] - ps)) < 2e-5


# ---------------------------------------------------------------------------
# full size (30 qubits, the bench's launch configuration): sampled outputs
# ---------------------------------------------------------------------------
def _qft_product_closed_form(us, n, k):
    # input psi_x = prod_q u_q[x_q]; QFT output at k = prod_q (u_q[0] + u_q[1] e^{2 pi i k / 2^(q+1)}) / sqrt 2
    out = np.ones(len(k), dtype=np.complex128)
    for q in range(n):
        out *= (us[q][0] + us[q][1] * np.exp(2j * np.pi * (k % (1 << (q + 1))) / (1 << (q + 1)))) / np.sqrt(2)
    return out


@pytest.mark.parametrize("mode", ["fused", "pergate"])
def test_qft30_full_size_sampled(mode):
    n = 30
    rng = np.random.default_rng(44)
    haar = [W.haar_u2(rng) for _ in range(n)]
    gl = [W.Gate("U", (q,), (), haar[q]) for q in range(n)] + W.qft_gates(n, swaps=True)
    st = qs.State(n)
    st.apply(gl, mode=mode)
    k = np.concatenate([np.arange(64), rng.integers(0, 1 << n, 4096), (1 << n) - 1 - np.arange(64)])
    got = st.tensor[0, torch.from_numpy(k).cuda()].cpu().numpy().astype(np.complex128)
    norm = float(torch.linalg.vector_norm(st.tensor[0]).item())
    st.close()
    ref = _qft_product_closed_form([h[:, 0] for h in haar], n, k)
    assert np.max(np.abs(got - ref)) <= 2e-5
    assert abs(norm - 1) < 1e-5


def test_tfim30_full_size_properties():
    n = 30
    gl = W.tfim_gates(n, 4, 0.05, 1.0, W.tfim_fields(n, 3), order=2)
    st = qs.State(n)
    st.apply(gl)
    a = st.tensor[0].clone()
    st.zero()
    st.apply(gl, mode="pergate")
    b = st.tensor[0]
    diff = float(torch.max(torch.abs(a - b)).item())
    norm = float(torch.linalg.vector_norm(a).item())
    st.close()
    assert abs(norm - 1) < 1e-5
    assert diff <= 2e-5   # both paths in complex64; the stated amplitude tolerance


@pytest.mark.parametrize("n,degree", [(16, 3), (22, 6), (22, 14)])
def test_factored_diagonals_in_layer_sweeps(n, degree):
    # random-angle ZZ couplings of the given degree interleaved with RX / RY
    # layers on scattered qubits: the diagonals' register groups span several
    # slice tables, which the planner factors per sweep (MK_DIAGQ) while each
    # group bit has at most 16 couplings, and keeps the general path above
    rng = np.random.default_rng(100 + n + degree)
    gl = []
    for layer in range(3):
        for i in range(n):
            for j in rng.choice(n, size=degree, replace=False):
                if i < j:
                    gl.append(W.Gate("RZZ", (i, int(j)), (float(rng.uniform(0, 2 * np.pi)),)))
        for q in rng.choice(n, size=n // 2, replace=False):
            gl.append(W.Gate("RX" if layer % 2 else "RY", (int(q),), (float(rng.uniform(0, 6)),)))
    psi0 = W.random_state(n, 9)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))
    _assert_close(_run(n, gl, psi0, dense="tf32x3"), _ref(n, gl, psi0))


@pytest.mark.parametrize("n", [9, 18])
def test_heisenberg_layers_basis_conjugated(n):
    # XXZ / random-field Heisenberg steps as same-family layers: each RXX run
    # becomes H (x) ZZ-phases (x) H and each RYY run (SH) ZZ (SH)^dagger
    # (Sec. 5.1 basis conjugation); plus single RXX / RYY gates that stay 4x4
    rng = np.random.default_rng(40 + n)
    gl = []
    for step in range(4):
        gl += [W.Gate("RXX", (i, i + 1), (float(rng.uniform(-1, 1)),)) for i in range(n - 1)]
        gl += [W.Gate("RYY", (i, i + 1), (float(rng.uniform(-1, 1)),)) for i in range(n - 1)]
        gl += [W.Gate("RZZ", (i, i + 1), (float(rng.uniform(-1, 1)),)) for i in range(n - 1)]
        gl += [W.Gate("RZ", (q,), (float(rng.uniform(-1, 1)),)) for q in range(n)]
        gl += [W.Gate("RXX", (0, n - 1), (0.3,)), W.Gate("H", (n // 2,)), W.Gate("RYY", (1, n - 2), (0.7,))]
    psi0 = W.random_state(n, 41)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))


def test_suite28_full_size_one_layer_and_full_suite():
    # the 28q layered suite at full size, in the launch configuration the
    # benchmark times: one layer (Haar U(2) on every qubit, CNOT ladder,
    # random ZZ bonds) from a Haar product state against the oracle's full
    # state; then 20 layers + QFT + WHT, fused against the per-gate path (norm
    # and relative L2: after 20 layers every amplitude is ~2^-14)
    n = 28
    rng = np.random.default_rng(28)
    vs = [W.haar_u2(rng)[:, 0] for _ in range(n)]
    hi, lo = vs[0], vs[n // 2]
    for v in vs[1:n // 2]:
        hi = np.kron(hi, v)
    for v in vs[n // 2 + 1:]:
        lo = np.kron(lo, v)
    psi0 = np.outer(hi, lo).reshape(-1).astype(np.complex64)
    del hi, lo
    gl = W.suite28_gates(n, 1, 5, tail=False)
    st = qs.State(n)
    st.set(psi0)
    st.apply(gl)
    got = st.get()[0]
    ref = oracle.simulate(n, gl, psi0.astype(np.complex128))
    _assert_close(got, ref)
    del got, ref
    suite = qs.CGates(W.suite28_gates(n, 20, 1, tail=True))
    st.set(psi0)
    st.apply(suite)
    a = st.tensor[0].clone()
    st.set(psi0)
    st.apply(suite, mode="pergate")
    b = st.tensor[0]
    rel = float((torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item())
    norm = float(torch.linalg.vector_norm(a).item())
    st.close()
    assert abs(norm - 1) < 1e-5
    assert rel <= 1e-5, rel


@pytest.mark.parametrize("n", [14, 22])
def test_count_table_diagonals(n):
    # uniform pair sums as count lookups: a ZZ chain and a ZZ random 3-regular
    # graph (mismatch counts), a CZ ring and a CP clique on 5 qubits inside one
    # register group (both-set counts, Qc up to 10), each with a uniform
    # single-qubit phase on some qubits, between RY / RX layers
    rng = np.random.default_rng(n)
    g = W.random_regular3_graph(n, rng)
    gl = [W.Gate("RY", (q,), (float(rng.uniform(0, 6)),)) for q in range(n)]
    gl += [W.Gate("RZZ", (b, b + 1), (0.37,)) for b in range(n - 1)]
    gl += [W.Gate("RX", (q,), (float(rng.uniform(0, 6)),)) for q in range(n)]
    gl += [W.Gate("RZZ", (u, v), (-0.81,)) for u, v in g] + [W.Gate("RZ", (q,), (0.29,)) for q in range(0, n, 3)]
    gl += [W.Gate("RY", (q,), (float(rng.uniform(0, 6)),)) for q in range(n)]
    gl += [W.Gate("CZ", (b, (b + 1) % n)) for b in range(n)] + [W.Gate("S", (q,)) for q in range(1, n, 2)]
    gl += [W.Gate("RX", (q,), (float(rng.uniform(0, 6)),)) for q in range(n)]
    gl += [W.Gate("CP", (i, j), (1.1,)) for i in range(n - 5, n) for j in range(i + 1, n)]
    gl += [W.Gate("RY", (q,), (float(rng.uniform(0, 6)),)) for q in range(n)]
    text, _ = qs.plan_describe(n, gl)
    assert "DIAGC=" in text, text
    psi0 = W.random_state(n, 5)
    _assert_close(_run(n, gl, psi0), _ref(n, gl, psi0))


def test_tile_pipeline_deterministic_across_autotune_shapes():
    # the 30q TFIM (10 Strang steps) under every shape the autotuner tries,
    # back to back on one state as the autotuner runs them: each shape applied
    # three times from the same input gives bit-identical states (a race in
    # the tile pipeline shows up as a difference), and the shapes agree with
    # one another to float rounding; the norm stays 1
    n = 30
    gl = qs.CGates(W.tfim_gates(n, 10, 0.05, 1.0, W.tfim_fields(n, 3), order=2))
    st = qs.State(n)
    st.provide_scratch()
    idx = torch.arange(0, 1 << n, 4099, device="cuda")
    ref = None
    for T, L, R in [(0, 0, 0), (12, 4, 4), (12, 4, 5), (12, 5, 4), (12, 5, 5), (13, 4, 4), (13, 4, 5),
                    (13, 5, 4), (13, 5, 5)]:
        outs = []
        for _ in range(3):
            st.zero()
            st.apply(gl, tile_qubits=T, low_qubits=L, group_qubits=R)
            outs.append(st.tensor[0][idx].clone())
        for o in outs[1:]:
            assert torch.equal(o, outs[0]), (T, L, R)
        assert abs(float(torch.linalg.vector_norm(st.tensor[0]).item()) - 1) < 1e-5
        if ref is None:
            ref = outs[0]
        else:
            d = float((outs[0] - ref).abs().max().item())
            assert d < 2e-6, (T, L, R, d)
    st.close()


@pytest.mark.parametrize("n,n_rand", [(24, 24), (28, 4)])
def test_expectation_reduction_error_against_oracle(n, n_rand):
    # qs_expect sums up to 64 FP32 products per thread before folding them into
    # FP64 (FP64 from the first product would cost several times the read on
    # this part).  Both sides read the same complex64 amplitudes (the oracle in
    # complex128), so the difference is the reduction's arithmetic alone: FP32
    # products (relative error 2^-24) and runs of <= 64 FP32 adds (typically
    # sqrt(64) 2^-24 relative), FP64 beyond: measured ~2e-11 of sum |c_k| at
    # n = 24 and ~1e-11 at n = 28.  The bound, 1e-9 of sum |c_k|, fails for a
    # reduction that keeps long FP32 sums (over 2^24 amplitudes they drift to
    # ~1e-7 relative).
    rng = np.random.default_rng(n)
    psi = W.random_state(n, 300 + n).astype(np.complex64)
    terms = W.tfim_paulis(n, 1.0, 0.7)
    terms += [(float(rng.normal()), int(rng.integers(1 << n)), int(rng.integers(1 << n))) for _ in range(n_rand)]
    st = qs.State(n)
    st.set(psi)
    got = st.expect(terms)[0]
    st.close()
    ref = oracle.expect(psi.astype(np.complex128), n, terms)
    scale = sum(abs(t[0]) for t in terms)
    err = abs(got - ref)
    print(f"n={n}: |<H>_gpu - <H>_oracle| = {err:.3e} = {err / scale:.3e} of sum|c|")
    assert err <= 1e-9 * scale, (got, ref, err / scale)
