"""GPU parity of the end-to-end sweep's workloads (the paper's gate-based
suite) at 16 qubits, fused path against the complex128 oracle, plus long
circuits on states that fit one tile (every pass ends at the builder's
sweep or micro-op limit and the rest carries over to the next pass).

Tolerance: relative L2 <= 1e-4 (up to ~10^3 complex64 roundings per
amplitude in the longest families), fidelity >= 1 - 1e-6."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_19147_gb300 as qs  # noqa: E402

N = 16
FAMILIES = W.sweep_workloads(N)


def _check(n, gates, seed, **kw):
    psi0 = W.random_state(n, seed)
    st = qs.State(n)
    st.set(psi0.astype(np.complex64))
    st.apply(gates, **kw)
    got = st.get()[0].astype(np.complex128)
    st.close()
    ref = oracle.simulate(n, gates, psi0.astype(np.complex64).astype(np.complex128))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real)
    return rel, fid


@pytest.mark.parametrize("idx", range(len(FAMILIES)), ids=[f[0] for f in FAMILIES])
def test_sweep_family_matches_oracle(idx):
    name, gates = FAMILIES[idx]
    rel, fid = _check(N, gates, 40 + idx)
    assert rel <= 1e-4 and fid >= 1 - 1e-6, (name, rel, fid)


@pytest.mark.parametrize("n,steps,kw", [(12, 40, {}), (13, 20, {"tile_qubits": 13, "group_qubits": 4})])
def test_long_single_tile_tfim(n, steps, kw):
    gates = W.tfim_gates(n, steps, 0.05, 1.0, W.tfim_fields(n, 11), order=2)
    rel, fid = _check(n, gates, 5, **kw)
    assert rel <= 1e-4 and fid >= 1 - 1e-6, (rel, fid)
