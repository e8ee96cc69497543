"""Full-size parity against the complex128 oracle, in the launch
configuration the benchmark times.

* The 28-qubit layered suite: 20 layers of Haar U(2) on every qubit, the
  ascending CNOT ladder and random-angle ZZ bonds, then the full-register QFT
  (with its swaps) and Walsh-Hadamard transform, applied by the fused path
  and by the oracle (one gate at a time on a 4 GiB complex128 state) from
  the same Haar product state, compared element by element.
* The 30-qubit gate-stream QFT (480 gates, with swaps) on a seeded random
  state against sqrt(N) * ifft of the complex128 input: the oracle's own
  QFT is pinned to that library routine (tests/test_oracle_pins.py), which
  stands in for 480 oracle gates on a 16 GiB state.

Tolerances as in the other parity tests: max |d amplitude| <= 2e-5, relative
L2 <= 1e-5, fidelity >= 1 - 1e-6.  These tests hold up to ~60 GB of host
memory and take a few minutes of host time.
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


def _compare(got, ref):
    # chunked so that no complex128 copy of the whole GPU result is made
    dmax, dd, rr, dot = 0.0, 0.0, 0.0, 0.0 + 0.0j
    gg = 0.0
    step = 1 << 24
    for i in range(0, ref.size, step):
        g = got[i:i + step].astype(np.complex128)
        r = ref[i:i + step]
        d = g - r
        dmax = max(dmax, float(np.max(np.abs(d))))
        dd += float(np.vdot(d, d).real)
        rr += float(np.vdot(r, r).real)
        gg += float(np.vdot(g, g).real)
        dot += complex(np.vdot(r, g))
    rel = (dd / rr) ** 0.5
    fid = abs(dot) ** 2 / (gg * rr)
    return dmax, rel, fid


def _haar_product_state(n, seed):
    rng = np.random.default_rng(seed)
    vs = [W.haar_u2(rng)[:, 0] for _ in range(n)]
    hi, lo = vs[0], vs[n // 2]
    for v in vs[1:n // 2]:
        hi = np.kron(hi, v)
    for v in vs[n // 2 + 1:]:
        lo = np.kron(lo, v)
    return np.outer(hi, lo).reshape(-1).astype(np.complex64)


def test_suite28_twenty_layers_qft_wht_against_oracle():
    n = 28
    psi0 = _haar_product_state(n, 28)
    gl = W.suite28_gates(n, 20, 1, tail=True)
    st = qs.State(n)
    st.set(psi0)
    st.apply(gl)
    got = st.get()[0]
    st.close()
    ref = oracle.simulate(n, gl, psi0.astype(np.complex128))
    del psi0
    d, rel, fid = _compare(got, ref)
    assert d <= 2e-5, d
    assert rel <= 1e-5, rel
    assert fid >= 1 - 1e-6, fid


def test_qft30_random_state_against_scaled_ifft():
    scipy_fft = pytest.importorskip("scipy.fft")
    n = 30
    psi0 = W.random_state(n, 4).astype(np.complex64)
    st = qs.State(n)
    st.set(psi0)
    st.apply(W.qft_gates(n, swaps=True))
    got = st.get()[0]
    st.close()
    ref = scipy_fft.ifft(psi0.astype(np.complex128), norm="ortho")   # sqrt(N) * ifft
    del psi0
    d, rel, fid = _compare(got, ref)
    assert d <= 2e-5, d
    assert rel <= 1e-5, rel
    assert fid >= 1 - 1e-6, fid
