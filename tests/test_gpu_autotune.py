"""The autotuner (qs_autotune): it leaves the state unchanged, returns one of
its candidate tile shapes, keeps the choice per gate structure (in memory and
in its cache file), and the chosen shape gives the oracle's result."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2609_19147_gb300 as qs  # noqa: E402

CANDIDATES = {(0, 0, 0)} | {(t, l, r) for t in (12, 13) for l in (4, 5) for r in (4, 5)}


def test_autotune_choice_cached_and_state_unchanged(tmp_path):
    n = 16
    gl = W.tfim_gates(n, 20, 0.05, 1.0, W.tfim_fields(n, 3), order=2)
    psi0 = W.random_state(n, 21).astype(np.complex64)
    st = qs.State(n)
    st.set(psi0)
    path = str(tmp_path / "tune.txt")
    cfg = st.autotune(gl, reps=1, cache_path=path)
    assert np.array_equal(st.get()[0], psi0)               # amplitudes untouched
    shape = (cfg["tile_qubits"], cfg["low_qubits"], cfg["group_qubits"])
    assert shape in CANDIDATES and cfg["ms"] > 0
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("qs-autotune ")
    # same structure, other angles: the kept choice, nothing re-timed
    gl2 = W.tfim_gates(n, 20, 0.07, 1.0, W.tfim_fields(n, 4), order=2)
    cfg2 = st.autotune(gl2, reps=1, cache_path=path)
    assert cfg2 == cfg
    assert len(open(path).read().splitlines()) == 1
    # the chosen shape reproduces the oracle
    kw = {k: v for k, v in cfg.items() if k != "ms"}
    st.apply(gl, **kw)
    got = st.get()[0].astype(np.complex128)
    st.close()
    ref = oracle.simulate(n, gl, psi0.astype(np.complex128))
    assert np.max(np.abs(got - ref)) <= 2e-5


def test_autotune_batched_params_and_bad_args():
    n, L, B = 14, 3, 4
    gl = W.vqe_ansatz_gates(n, L)
    theta = W.vqe_params(n, L, B, 9)
    st = qs.State(n, batch=B)
    cfg = st.autotune(gl, params=theta, reps=1)
    kw = {k: v for k, v in cfg.items() if k != "ms"}
    st.apply(gl, params=theta, **kw)
    got = st.get()
    for b in range(B):
        ref = oracle.simulate(n, gl, theta=theta[b])
        assert np.max(np.abs(got[b].astype(np.complex128) - ref)) <= 2e-5
    with pytest.raises(qs.QsError):
        st.autotune(gl, params=theta, reps=0)
    st.close()
