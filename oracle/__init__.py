"""The oracle: a plain, slow, complex128 CPU state-vector simulator.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
bench's ``cpu_baseline`` / ``--impl reference`` legs may import it.  The CUDA
path (``paper_2609_19147_gb300``) neither imports it nor shares code with it;
both read their inputs from ``workloads``.

What it computes: the result of applying a gate list one gate at a time, in
order, to a complex128 state (Sec. 2.1 state-vector simulation; Sec. 3.2.2 gate
application and gate library).  Every fused layer family of Sec. 5.1 (phase-LUT
diagonals, GF(2) gathers, tensor-product 1-qubit layers, radix-4 QFT / Walsh
butterflies, basis-conjugated XX/YY layers) reaches exactly this result up to
rounding order, so this per-gate definition is the oracle for all of them.
Expectation values follow the Pauli-observable capability of Sec. 3.2.1 and
gradients the parameter-shift rule of Sec. 3.2.3 (hardware-efficient ansatz).

Pins (tests/test_oracle_*.py): textbook gate identities and expm of the
generators; an independent einsum / full-matrix simulator for n <= 8
(oracle.brute); QFT vs the normalised DFT column and sqrt(N) ifft; GHZ; WHT
twice = I; Grover's sin^2((2k+1) theta); the first-order TFIM Trotter-error
table printed in Sec. 6.4 (tests/golden); second-order error scaling vs exact
diagonalisation; parameter shift vs finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Iterable, Optional, Sequence

import numpy as np

from . import gates as _g

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile sv.c into a shared library with gcc/OpenMP (portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_apply.restype = ctypes.c_int
        lib.orc_apply.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
        lib.orc_vdot.restype = None
        lib.orc_vdot.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_set_threads.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(t: int) -> None:
    """Thread count of the C core's parallel loops (for timing)."""
    _load().orc_set_threads(int(t))


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_matrix(psi: np.ndarray, n: int, wires: Sequence[int], U: np.ndarray) -> None:
    """In place: apply the k-qubit matrix U to `wires` (first wire = MSB of U's index)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == (1 << n)
    k = len(wires)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    assert U.shape == (1 << k, 1 << k)
    w = (ctypes.c_int * k)(*[int(x) for x in wires])
    rc = _load().orc_apply(n, psi.ctypes.data, k, w, U.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle rejected gate on wires {wires} for n={n}")


def gate_matrix(g) -> np.ndarray:
    return _g.matrix(g.kind, g.params, g.matrix)


def apply_gates(psi: np.ndarray, n: int, gate_list: Iterable, theta: Optional[np.ndarray] = None) -> np.ndarray:
    """Apply each gate in order (in place).  `theta` resolves parameter indices."""
    for g in gate_list:
        params = g.params
        if theta is not None and g.pidx >= 0:
            params = (float(theta[g.pidx]),) + tuple(g.params[1:])
        apply_matrix(psi, n, g.wires, _g.matrix(g.kind, params, g.matrix))
    return psi


def simulate(n: int, gate_list: Iterable, psi0: Optional[np.ndarray] = None,
             theta: Optional[np.ndarray] = None) -> np.ndarray:
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128, copy=True)
    return apply_gates(psi, n, gate_list, theta)


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_vdot(a.size, a.ctypes.data, b.ctypes.data, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def apply_pauli(psi: np.ndarray, n: int, x_mask: int, z_mask: int) -> np.ndarray:
    """Return P psi for the Pauli string with bit q of the masks = qubit q
    (X where only x is set, Z where only z, Y where both)."""
    out = psi.copy()
    for q in range(n):
        xb, zb = (x_mask >> q) & 1, (z_mask >> q) & 1
        if xb or zb:
            c = "Y" if (xb and zb) else ("X" if xb else "Z")
            apply_matrix(out, n, (q,), _g.pauli(c))
    return out


def expect(psi: np.ndarray, n: int, terms) -> float:
    """<psi| sum_k c_k P_k |psi> for a Hermitian Pauli sum (real result)."""
    tot = 0.0 + 0.0j
    for (c, xm, zm) in terms:
        if xm == 0 and zm == 0:
            tot += c * vdot(psi, psi)
        else:
            tot += c * vdot(psi, apply_pauli(psi, n, xm, zm))
    return float(tot.real)


def energy(n: int, gate_list, theta: np.ndarray, terms) -> float:
    return expect(simulate(n, gate_list, theta=theta), n, terms)


def param_shift_grad(n: int, gate_list, theta: np.ndarray, terms,
                     indices: Optional[Sequence[int]] = None) -> np.ndarray:
    """dE/dtheta_i = [E(theta + pi/2 e_i) - E(theta - pi/2 e_i)] / 2, exact for
    gates exp(-i theta G / 2) with G^2 = I when theta_i enters one gate."""
    theta = np.asarray(theta, dtype=np.float64)
    idx = list(range(theta.size)) if indices is None else list(indices)
    out = np.zeros(len(idx))
    for j, i in enumerate(idx):
        tp = theta.copy()
        tp[i] += np.pi / 2
        tm = theta.copy()
        tm[i] -= np.pi / 2
        out[j] = 0.5 * (energy(n, gate_list, tp, terms) - energy(n, gate_list, tm, terms))
    return out


def finite_diff_grad(n: int, gate_list, theta: np.ndarray, terms, eps: float = 1e-5,
                     indices: Optional[Sequence[int]] = None) -> np.ndarray:
    theta = np.asarray(theta, dtype=np.float64)
    idx = list(range(theta.size)) if indices is None else list(indices)
    out = np.zeros(len(idx))
    for j, i in enumerate(idx):
        tp = theta.copy()
        tp[i] += eps
        tm = theta.copy()
        tm[i] -= eps
        out[j] = (energy(n, gate_list, tp, terms) - energy(n, gate_list, tm, terms)) / (2 * eps)
    return out


def expected_cut(psi: np.ndarray, n: int, edges) -> float:
    """<C> = sum_x |psi_x|^2 cut(x), cut(x) = number of edges whose endpoint bits
    differ (Sec. 3.2.3 MaxCut cost), from the probabilities directly."""
    p = np.abs(psi) ** 2
    x = np.arange(1 << n, dtype=np.int64)
    cut = np.zeros(1 << n, dtype=np.int64)
    for (u, v) in edges:
        cut += ((x >> (n - 1 - u)) ^ (x >> (n - 1 - v))) & 1
    return float(np.dot(p, cut))
