"""Oracle gate matrices in complex128 (test infrastructure only).

Each matrix is the textbook definition of the gate named in the paper's gate
library (Sec. 3.2.2: Pauli, Clifford, rotation, U1/U2/U3, Toffoli, Fredkin;
Table "OpenQASM 2.0 gate coverage": S-dagger, T-dagger, SX, iSWAP, CH,
CRX/CRY/CRZ) and its layer families (Sec. 5.1: ZZ / XX / YY Trotter terms,
CPHASE).  Rotation convention: R_P(theta) = exp(-i theta P / 2); the RZZ
mapping theta = -2 J dt of Sec. 4.1 fixes RZZ(theta) = exp(-i theta/2 Z(x)Z).
Multi-qubit matrices are indexed with the first listed wire as the most
significant bit (controls first).

Only tests/, __graft_entry__.smoke() and the bench's CPU-baseline legs may use
this package; the CUDA path never imports it.
"""
from __future__ import annotations

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def pauli(c: str) -> np.ndarray:
    return {"I": _I2, "X": _X, "Y": _Y, "Z": _Z}[c].copy()


def _rot(P: np.ndarray, theta: float) -> np.ndarray:
    # exp(-i theta P / 2) for P^2 = I: cos(theta/2) I - i sin(theta/2) P
    return np.cos(theta / 2.0) * np.eye(P.shape[0]) - 1j * np.sin(theta / 2.0) * P


def _controlled(U: np.ndarray) -> np.ndarray:
    k = U.shape[0]
    M = np.eye(2 * k, dtype=np.complex128)
    M[k:, k:] = U
    return M


def matrix(kind: str, params=(), mat=None) -> np.ndarray:
    """Unitary of one gate record (complex128)."""
    p = tuple(float(x) for x in params)
    if kind == "I":
        return _I2.copy()
    if kind == "X":
        return _X.copy()
    if kind == "Y":
        return _Y.copy()
    if kind == "Z":
        return _Z.copy()
    if kind == "H":
        return _H.copy()
    if kind == "S":
        return np.diag([1, 1j]).astype(np.complex128)
    if kind == "SDG":
        return np.diag([1, -1j]).astype(np.complex128)
    if kind == "T":
        return np.diag([1, np.exp(1j * np.pi / 4)]).astype(np.complex128)
    if kind == "TDG":
        return np.diag([1, np.exp(-1j * np.pi / 4)]).astype(np.complex128)
    if kind == "SX":
        return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
    if kind == "RX":
        return _rot(_X, p[0])
    if kind == "RY":
        return _rot(_Y, p[0])
    if kind == "RZ":
        return _rot(_Z, p[0])
    if kind == "P":        # U1(lambda) = diag(1, e^{i lambda})
        return np.diag([1, np.exp(1j * p[0])]).astype(np.complex128)
    if kind == "U2":       # OpenQASM 2.0: U2(phi, lambda) = U3(pi/2, phi, lambda)
        return matrix("U3", (np.pi / 2, p[0], p[1]))
    if kind == "U3":       # OpenQASM 2.0 U(theta, phi, lambda)
        t, ph, la = p
        c, s = np.cos(t / 2), np.sin(t / 2)
        return np.array([[c, -np.exp(1j * la) * s],
                         [np.exp(1j * ph) * s, np.exp(1j * (ph + la)) * c]], dtype=np.complex128)
    if kind == "U":
        return np.asarray(mat, dtype=np.complex128).reshape(2, 2).copy()
    if kind == "CX":
        return _controlled(_X)
    if kind == "CY":
        return _controlled(_Y)
    if kind == "CZ":
        return _controlled(_Z)
    if kind == "CH":
        return _controlled(_H)
    if kind == "CRX":
        return _controlled(_rot(_X, p[0]))
    if kind == "CRY":
        return _controlled(_rot(_Y, p[0]))
    if kind == "CRZ":
        return _controlled(_rot(_Z, p[0]))
    if kind == "CP":       # CPHASE(theta) = diag(1, 1, 1, e^{i theta})
        return np.diag([1, 1, 1, np.exp(1j * p[0])]).astype(np.complex128)
    if kind == "SWAP":
        M = np.zeros((4, 4), dtype=np.complex128)
        M[0, 0] = M[1, 2] = M[2, 1] = M[3, 3] = 1
        return M
    if kind == "ISWAP":
        M = np.zeros((4, 4), dtype=np.complex128)
        M[0, 0] = M[3, 3] = 1
        M[1, 2] = M[2, 1] = 1j
        return M
    if kind == "RZZ":
        return _rot(np.kron(_Z, _Z), p[0])
    if kind == "RXX":
        return _rot(np.kron(_X, _X), p[0])
    if kind == "RYY":
        return _rot(np.kron(_Y, _Y), p[0])
    if kind == "CCX":
        return _controlled(_controlled(_X))
    if kind == "CSWAP":
        return _controlled(matrix("SWAP"))
    raise ValueError(f"unknown gate kind {kind!r}")


# generator G of each parametric gate R(theta) = exp(-i theta G / 2), used by
# the parameter-shift rule (G^2 = I, so the shift is +-pi/2)
def generator(kind: str) -> np.ndarray:
    return {"RX": _X, "RY": _Y, "RZ": _Z, "RZZ": np.kron(_Z, _Z),
            "RXX": np.kron(_X, _X), "RYY": np.kron(_Y, _Y)}[kind].copy()
