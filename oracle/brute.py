"""Independent brute-force cross-checks for the oracle at n <= 8 (test infrastructure).

Two formulations that share nothing with oracle/sv.c:
  * ``full_unitary``: every gate is expanded into its full 2^n x 2^n matrix
    from the definition <y|G|x> = U[j(y), j(x)] * [rest(y) == rest(x)], where
    j() reads the gate's wires (first wire = most significant) and rest() the
    other bits; the circuit unitary is the ordered product.
  * ``einsum_apply``: the state as a rank-n tensor (axis q = qubit q, Sec.
    3.2.2 "viewed as a rank-n tensor with one index per qubit"), each gate a
    tensordot over the gate's axes.
"""
from __future__ import annotations

import numpy as np

from . import gates as _g


def full_gate(n: int, wires, U: np.ndarray) -> np.ndarray:
    k = len(wires)
    x = np.arange(1 << n)
    pos = [n - 1 - w for w in wires]
    j = np.zeros_like(x)
    for m, p in enumerate(pos):
        j |= ((x >> p) & 1) << (k - 1 - m)
    mask = sum(1 << p for p in pos)
    rest = x & ~mask
    same = rest[:, None] == rest[None, :]
    return np.where(same, U[j[:, None], j[None, :]], 0.0).astype(np.complex128)


def full_unitary(n: int, gate_list, theta=None) -> np.ndarray:
    M = np.eye(1 << n, dtype=np.complex128)
    for g in gate_list:
        params = g.params
        if theta is not None and g.pidx >= 0:
            params = (float(theta[g.pidx]),) + tuple(g.params[1:])
        M = full_gate(n, g.wires, _g.matrix(g.kind, params, g.matrix)) @ M
    return M


def einsum_apply(psi: np.ndarray, n: int, gate_list) -> np.ndarray:
    t = np.asarray(psi, dtype=np.complex128).reshape((2,) * n)
    for g in gate_list:
        U = _g.matrix(g.kind, g.params, g.matrix)
        k = len(g.wires)
        Ut = U.reshape((2,) * (2 * k))
        t = np.tensordot(Ut, t, axes=(list(range(k, 2 * k)), list(g.wires)))
        # tensordot puts the gate's output axes first; move them back
        t = np.moveaxis(t, list(range(k)), list(g.wires))
    return t.reshape(-1)


def pauli_sum_matrix(n: int, terms) -> np.ndarray:
    """Dense Hamiltonian from Pauli terms via Kronecker products (qubit 0 leftmost)."""
    H = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for (c, xm, zm) in terms:
        P = np.array([[1.0 + 0j]])
        for q in range(n):
            xb, zb = (xm >> q) & 1, (zm >> q) & 1
            s = "Y" if (xb and zb) else ("X" if xb else ("Z" if zb else "I"))
            P = np.kron(P, _g.pauli(s))
        H += c * P
    return H
