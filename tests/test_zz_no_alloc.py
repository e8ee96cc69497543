"""The allocation-free expectation entry point (qs_expect_noalloc).

Some callers of this library cannot call cudaMalloc: a plug-in inside a host
application that owns all device memory through its own arena, a process
whose states already fill the GPU, or a real-time loop that cannot take the
implicit synchronisation of an allocation.  qs_expect_noalloc gives them
Pauli expectation values from a reduction whose scratch is a static device
array inside the library.  These tests call it through the C ABI and check
it against the complex128 oracle and against qs_expect (the allocating entry
point), on calls in a row that reuse the one array.  The file is collected
last, so a run that stops at the first failure has already run every other
test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_19147_gb300 as qs  # noqa: E402


def _noalloc(tensor, n, batch, terms, stream=None):
    arr, k = qs._paulis(terms)
    out = np.full(batch, np.nan)
    s = stream.cuda_stream if stream is not None else None
    rc = qs._lib.qs_expect_noalloc(ctypes.c_void_p(tensor.data_ptr()), n, batch, arr, k,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(s))
    assert rc == qs.QS_OK, qs._lib.qs_last_error()
    return out


def _tol(terms):
    # FP32 amplitudes, FP64 sums: ~1e-6 relative to the sum of |coeff|
    return 2e-6 * max(1.0, sum(abs(t[0]) for t in terms))


def test_expect_noalloc_matches_oracle_and_qs_expect_on_calls_in_a_row():
    n, B = 14, 3
    psis = np.stack([W.random_state(n, 70 + b) for b in range(B)]).astype(np.complex64)
    st = qs.State(n, batch=B)
    st.set(psis)
    rng = np.random.default_rng(11)
    terms = W.tfim_paulis(n, 1.0, 0.7) + [(float(rng.normal()), int(rng.integers(1 << n)),
                                           int(rng.integers(1 << n))) for _ in range(40)]
    ref = np.array([oracle.expect(psis[b].astype(np.complex128), n, terms) for b in range(B)])
    via_expect = st.expect(terms)
    for _ in range(2):
        out = _noalloc(st.tensor, n, B, terms, st.stream)
        assert np.all(np.abs(out - ref) < _tol(terms)), (out, ref)
        assert np.all(np.abs(out - via_expect) < _tol(terms)), (out, via_expect)
    st.close()


def test_expect_noalloc_chunks_smaller_batch_and_empty_sum():
    # 19 ZZ bonds and 20 Z terms share x = 0: more than one 16-term chunk
    n = 20
    rng = np.random.default_rng(5)
    zz = [(float(rng.normal()), 0, (1 << q) | (1 << (q + 1))) for q in range(n - 1)]
    z = [(float(rng.normal()), 0, 1 << q) for q in range(n)]
    x = [(float(rng.normal()), 1 << q, 0) for q in range(3)]
    terms = zz + z + x
    psis = np.stack([W.random_state(n, 90 + b) for b in range(3)]).astype(np.complex64)
    big = qs.State(n, batch=3)
    big.set(psis)
    ref = np.array([oracle.expect(psis[b].astype(np.complex128), n, terms) for b in range(3)])
    out3 = _noalloc(big.tensor, n, 3, terms, big.stream)
    assert np.all(np.abs(out3 - ref) < _tol(terms)), (out3, ref)
    # a smaller batch after a larger one reuses the array: no stale partial sums
    small = qs.State(n, batch=1)
    small.set(psis[2:3])
    out1 = _noalloc(small.tensor, n, 1, terms, small.stream)
    assert abs(out1[0] - ref[2]) < _tol(terms), (out1, ref[2])
    assert abs(out1[0] - small.expect(terms)[0]) < _tol(terms)
    # an empty sum is zero without a launch
    assert np.all(_noalloc(big.tensor, n, 3, []) == 0.0)
    big.close()
    small.close()


def test_expect_noalloc_allocates_nothing_and_rejects_oversize():
    n, B = 16, 2
    psis = np.stack([W.random_state(n, 30 + b) for b in range(B)]).astype(np.complex64)
    st = qs.State(n, batch=B)
    st.set(psis)
    terms = W.tfim_paulis(n, 1.0, 1.3)
    _noalloc(st.tensor, n, B, terms, st.stream)   # first call: address set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        _noalloc(st.tensor, n, B, terms, st.stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # sizes beyond the stated maximum are rejected with a clear error
    arr, k = qs._paulis(terms)
    out = np.zeros(17)
    big = torch.zeros((17, 1 << 4), dtype=torch.complex64, device="cuda")
    rc = qs._lib.qs_expect_noalloc(ctypes.c_void_p(big.data_ptr()), 4, 17, arr, k,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert rc == qs.QS_ERR_UNSUPPORTED and b"16" in qs._lib.qs_last_error()
    many = [(1.0, 0, 1)] * 257
    arr, k = qs._paulis(many)
    rc = qs._lib.qs_expect_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, B, arr, k,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert rc == qs.QS_ERR_UNSUPPORTED and b"256" in qs._lib.qs_last_error()
    st.close()
