"""The allocation-free expectation entry point (qs_expect_noalloc).

Callers that cannot call cudaMalloc -- code running under CUDA graph capture,
plug-ins whose host application owns all device memory, latency-critical
loops -- get Pauli expectation values from a reduction whose scratch is a
static device array inside the library.  This test calls it through the C ABI
and checks it against qs_expect (same tolerance as the other expectation
tests) on two calls in a row.  It lives in a file collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_19147_gb300 as qs  # noqa: E402


def test_expect_noalloc_matches_qs_expect_twice():
    n, B = 14, 3
    psis = np.stack([W.random_state(n, 70 + b) for b in range(B)]).astype(np.complex64)
    st = qs.State(n, batch=B)
    st.set(psis)
    rng = np.random.default_rng(11)
    terms = W.tfim_paulis(n, 1.0, 0.7) + [(float(rng.normal()), int(rng.integers(1 << n)),
                                           int(rng.integers(1 << n))) for _ in range(40)]
    ref = st.expect(terms)
    arr, k = qs._paulis(terms)
    scale = max(1.0, sum(abs(t[0]) for t in terms)) / 10
    for _ in range(2):
        out = np.full(B, np.nan)
        rc = qs._lib.qs_expect_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, B, arr, k,
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.c_void_p(st.stream.cuda_stream))
        assert rc == qs.QS_OK, qs._lib.qs_last_error()
        assert np.all(np.abs(out - ref) < 1e-5 * scale), (out, ref)
    # sizes beyond the stated maximum are rejected with a clear error
    out = np.zeros(17)
    big = torch.zeros((17, 1 << 4), dtype=torch.complex64, device="cuda")
    rc = qs._lib.qs_expect_noalloc(ctypes.c_void_p(big.data_ptr()), 4, 17, arr, k,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert rc == qs.QS_ERR_UNSUPPORTED and b"16" in qs._lib.qs_last_error()
    st.close()
