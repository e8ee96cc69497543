"""Seeded synthetic inputs shared by the CUDA path (tests, bench) and the oracle.

This module holds gate *lists* (gate names, wires, angles), random states,
Haar-random U(2) draws, random graphs and Pauli-sum descriptions.  It holds
none of the simulator's arithmetic: no gate matrix is built here (except the
Haar draws, which are random inputs the method consumes), and no state is
evolved.  Both the CUDA binding and the oracle translate these records into
their own representations.

Conventions (stated once, used by every generator):
  * qubit q is bit n-1-q of the basis index (most significant first; the
    paper's reshape of the state as (2^q, 2, 2^(n-q-1)) in Sec. 3.2.2 and App. A).
  * Two-qubit gate records list wires in matrix order: the first wire is the
    more significant bit of the gate's 4x4 index (control first for
    controlled gates).
  * Pauli terms are (coeff, x_mask, z_mask) with bit q of a mask = qubit q;
    a qubit with both bits set carries Y.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Gate vocabulary (Sec. 3.2.2 gate library; Table "OpenQASM 2.0 gate coverage";
# Sec. 5.1 layer families add RZZ/RXX/RYY).
ONE_QUBIT = ("I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "SX",
             "RX", "RY", "RZ", "P", "U2", "U3", "U")
TWO_QUBIT = ("CX", "CY", "CZ", "CH", "SWAP", "ISWAP", "CRX", "CRY", "CRZ",
             "CP", "RZZ", "RXX", "RYY")
THREE_QUBIT = ("CCX", "CSWAP")
N_PARAMS = {"RX": 1, "RY": 1, "RZ": 1, "P": 1, "U2": 2, "U3": 3,
            "CRX": 1, "CRY": 1, "CRZ": 1, "CP": 1, "RZZ": 1, "RXX": 1, "RYY": 1}
PARAMETRIC = ("RX", "RY", "RZ", "RZZ", "CP")


@dataclass
class Gate:
    kind: str
    wires: Tuple[int, ...]
    params: Tuple[float, ...] = ()
    matrix: Optional[np.ndarray] = None     # only for kind "U": 2x2 complex128
    pidx: int = -1                          # parameter index (params[0] taken from a vector)


def arity(kind: str) -> int:
    if kind in ONE_QUBIT:
        return 1
    if kind in TWO_QUBIT:
        return 2
    if kind in THREE_QUBIT:
        return 3
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# random inputs
# ----------------------------------------------------------------------------
def random_state(n: int, seed: int) -> np.ndarray:
    """iid N(0,1) real and imaginary parts, normalised in FP64 (complex128)."""
    rng = np.random.default_rng(seed)
    dim = 1 << n
    psi = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    psi /= np.linalg.norm(psi)
    return psi


def haar_u2(rng: np.random.Generator) -> np.ndarray:
    """One Haar-random 2x2 unitary: QR of a complex Ginibre matrix with the
    phases of R's diagonal moved into Q (Mezzadri 2007)."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_regular3_graph(n: int, rng: np.random.Generator) -> List[Tuple[int, int]]:
    """Random simple 3-regular graph on n (even) vertices: pairing model with
    rejection of self-loops and repeated edges."""
    if n % 2:
        raise ValueError("3-regular graphs need an even vertex count")
    while True:
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)


# ----------------------------------------------------------------------------
# circuits
# ----------------------------------------------------------------------------
def qft_gates(n: int, swaps: bool = True) -> List[Gate]:
    """Gate-stream QFT (Sec. 3.2.3 QFT definition; Sec. 4 workloads).
    For qubit j = 0..n-1: H(j), then CP(j, k, pi/2^(k-j)) for k = j+1..n-1;
    then SWAP(j, n-1-j) for j < n/2 when `swaps`."""
    g: List[Gate] = []
    for j in range(n):
        g.append(Gate("H", (j,)))
        for k in range(j + 1, n):
            g.append(Gate("CP", (k, j), (np.pi / 2.0 ** (k - j),)))
    if swaps:
        for j in range(n // 2):
            g.append(Gate("SWAP", (j, n - 1 - j)))
    return g


def wht_gates(n: int) -> List[Gate]:
    """Hadamard on every qubit (App. A)."""
    return [Gate("H", (q,)) for q in range(n)]


def ghz_gates(n: int) -> List[Gate]:
    """H on qubit 0 then the CNOT chain 0->1->...->n-1 (Sec. 3.2.3 GHZ)."""
    return [Gate("H", (0,))] + [Gate("CX", (q, q + 1)) for q in range(n - 1)]


def cnot_ladder(n: int) -> List[Gate]:
    """Ascending CNOT ladder i -> i+1, i = 0..n-2."""
    return [Gate("CX", (q, q + 1)) for q in range(n - 1)]


def suite28_gates(n: int, layers: int, seed: int, tail: bool = True) -> List[Gate]:
    """Layered suite: `layers` x [Haar U(2) on every qubit, ascending CNOT
    ladder, RZZ(theta_b) on bonds (i, i+1) with theta_b ~ U[0, 2pi) drawn per
    layer], then (if `tail`) a full-register QFT (with swaps) and a WHT."""
    rng = np.random.default_rng(seed)
    g: List[Gate] = []
    for _ in range(layers):
        for q in range(n):
            g.append(Gate("U", (q,), (), haar_u2(rng)))
        g.extend(cnot_ladder(n))
        thetas = rng.uniform(0.0, 2.0 * np.pi, size=n - 1)
        for b in range(n - 1):
            g.append(Gate("RZZ", (b, b + 1), (float(thetas[b]),)))
    if tail:
        g.extend(qft_gates(n, swaps=True))
        g.extend(wht_gates(n))
    return g


def tfim_fields(n: int, seed: int, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    """Per-site transverse fields h_i ~ U[lo, hi] (seeded)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def tfim_gates(n: int, steps: int, dt: float, J: float = 1.0, h=0.5,
               order: int = 1) -> List[Gate]:
    """TFIM product formula on an open chain, H = -J sum Z_i Z_{i+1} + sum h_i X_i
    (Sec. 3.2.3 Hamiltonian simulation).  e^{iJ ZZ dt} = RZZ(-2 J dt) and
    e^{-i h X dt} = RX(2 h dt).  order=1: [ZZ(dt) bonds, X(dt) sites] per step.
    order=2 (Strang): [ZZ(dt/2), X(dt), ZZ(dt/2)] per step."""
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    g: List[Gate] = []

    def zz(frac):
        for b in range(n - 1):
            g.append(Gate("RZZ", (b, b + 1), (-2.0 * J * dt * frac,)))

    def xx():
        for q in range(n):
            g.append(Gate("RX", (q,), (2.0 * float(hs[q]) * dt,)))

    for _ in range(steps):
        if order == 1:
            zz(1.0)
            xx()
        elif order == 2:
            zz(0.5)
            xx()
            zz(0.5)
        else:
            raise ValueError(order)
    return g


def grover_gates(n: int, marked: Sequence[int], iterations: int) -> List[Gate]:
    """Grover search from |0..0>: H on all, then `iterations` x [phase-flip
    oracle on each marked basis index, diffusion H^n (2|0><0| - I) H^n].
    The phase flip of index m is X on the zero bits of m, a multi-controlled Z
    realised as H-CCX-H ladders is avoided: this generator is only used for
    n <= 3 with CZ / Z / CCZ-by-H-conjugation patterns."""
    if n not in (2, 3):
        raise ValueError("grover_gates supports n = 2 or 3")
    g: List[Gate] = [Gate("H", (q,)) for q in range(n)]

    def mcz():
        if n == 2:
            g.append(Gate("CZ", (0, 1)))
        else:
            g.append(Gate("H", (2,)))
            g.append(Gate("CCX", (0, 1, 2)))
            g.append(Gate("H", (2,)))

    def flip_index(m):
        zeros = [q for q in range(n) if not (m >> (n - 1 - q)) & 1]
        for q in zeros:
            g.append(Gate("X", (q,)))
        mcz()
        for q in zeros:
            g.append(Gate("X", (q,)))

    for _ in range(iterations):
        for m in marked:
            flip_index(m)
        for q in range(n):
            g.append(Gate("H", (q,)))
        flip_index(0)          # -(2|0><0| - I) up to global phase -1
        for q in range(n):
            g.append(Gate("H", (q,)))
    return g


def qaoa_gates(n: int, edges: Sequence[Tuple[int, int]], gammas: Sequence[float],
               betas: Sequence[float]) -> List[Gate]:
    """QAOA MaxCut circuit (Sec. 3.2.3 QAOA): |+>^n prepared by H on all
    qubits, then for each layer e^{-i gamma H_C} as RZZ(-gamma) per edge
    (H_C = 1/2 sum (I - Z_u Z_v); the dropped factor is a global phase) and
    e^{-i beta H_M} as RX(2 beta) per qubit."""
    g: List[Gate] = [Gate("H", (q,)) for q in range(n)]
    for gam, bet in zip(gammas, betas):
        for (u, v) in edges:
            g.append(Gate("RZZ", (u, v), (-float(gam),)))
        for q in range(n):
            g.append(Gate("RX", (q,), (2.0 * float(bet),)))
    return g


def qaoa_batch(seed: int, n_graphs: int = 512, n_choices=(14, 16, 18, 20, 22, 24),
               p: int = 4, n_angle_sets: int = 8):
    """Batched QAOA instances: `n_graphs` random 3-regular graphs with n drawn
    uniformly from `n_choices`, each with `n_angle_sets` angle sets
    (gamma_1..p, beta_1..p) ~ U[0, pi).  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for gi in range(n_graphs):
        n = int(rng.choice(n_choices))
        edges = random_regular3_graph(n, rng)
        angles = rng.uniform(0.0, np.pi, size=(n_angle_sets, 2, p))
        out.append({"n": n, "edges": edges, "gammas": angles[:, 0, :], "betas": angles[:, 1, :]})
    return out


def maxcut_paulis(n: int, edges: Sequence[Tuple[int, int]]):
    """C = sum_edges (1 - Z_u Z_v)/2 as Pauli terms (coeff, x_mask, z_mask)."""
    terms = [(0.5 * len(edges), 0, 0)]
    for (u, v) in edges:
        terms.append((-0.5, 0, (1 << u) | (1 << v)))
    return terms


def tfim_paulis(n: int, J: float = 1.0, h: float = 1.0):
    """H = -J sum_{i<n-1} Z_i Z_{i+1} + h sum_i X_i (open chain) as Pauli terms."""
    terms = [(-J, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    terms += [(h, 1 << i, 0) for i in range(n)]
    return terms


def vqe_ansatz_gates(n: int, layers: int) -> List[Gate]:
    """Hardware-efficient ansatz: per layer RY(theta) on every qubit, RZ(phi) on
    every qubit, then CNOT(q -> q+1 mod n) for q = 0..n-1.  Parameter index of
    RY on (l, q) is 2(l n + q), of RZ is 2(l n + q) + 1.  Angles are taken from
    the parameter vector (pidx); the stored params are placeholders."""
    g: List[Gate] = []
    for l in range(layers):
        for q in range(n):
            g.append(Gate("RY", (q,), (0.0,), None, 2 * (l * n + q)))
        for q in range(n):
            g.append(Gate("RZ", (q,), (0.0,), None, 2 * (l * n + q) + 1))
        for q in range(n):
            g.append(Gate("CX", (q, (q + 1) % n)))
    return g


def vqe_params(n: int, layers: int, batch: int, seed: int) -> np.ndarray:
    """batch x (2 n layers) angles ~ U[0, 2pi)."""
    return np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, size=(batch, 2 * n * layers))


def random_circuit(n: int, n_gates: int, seed: int, kinds: Sequence[str] = None) -> List[Gate]:
    """Random gate list over the whole vocabulary (for parity and fusion tests)."""
    rng = np.random.default_rng(seed)
    kinds = list(kinds) if kinds is not None else list(ONE_QUBIT + TWO_QUBIT + THREE_QUBIT)
    kinds = [k for k in kinds if arity(k) <= n]
    g: List[Gate] = []
    for _ in range(n_gates):
        k = kinds[int(rng.integers(len(kinds)))]
        w = tuple(int(x) for x in rng.choice(n, size=arity(k), replace=False))
        params = tuple(float(x) for x in rng.uniform(-np.pi, np.pi, size=N_PARAMS.get(k, 0)))
        mat = haar_u2(rng) if k == "U" else None
        g.append(Gate(k, w, params, mat))
    return g


def bind_params(gates: Sequence[Gate], theta: np.ndarray) -> List[Gate]:
    """Resolve parameter indices: params[0] <- theta[pidx]."""
    out = []
    for gt in gates:
        if gt.pidx >= 0:
            p = (float(theta[gt.pidx]),) + tuple(gt.params[1:])
            out.append(Gate(gt.kind, gt.wires, p, gt.matrix, gt.pidx))
        else:
            out.append(gt)
    return out


def spell_out_2q(gates: Sequence[Gate]) -> List[Gate]:
    """The two-qubit diagonals written the way imported circuits often carry
    them (App. B.1: a QFT arriving as cx + rz / u1 sequences): CP(l) on
    (c, t) as P(l/2) c, CX(c, t), P(-l/2) t, CX(c, t), P(l/2) t; RZZ(t) on
    (a, b) as CX(a, b), RZ(t) b, CX(a, b); CZ as CP(pi); other gates as they are."""
    out: List[Gate] = []
    for g in gates:
        if g.kind in ("CP", "CZ"):
            c, t = g.wires
            lam = float(g.params[0]) if g.kind == "CP" else float(np.pi)
            out += [Gate("P", (c,), (lam / 2,)), Gate("CX", (c, t)), Gate("P", (t,), (-lam / 2,)),
                    Gate("CX", (c, t)), Gate("P", (t,), (lam / 2,))]
        elif g.kind == "RZZ":
            a, b = g.wires
            out += [Gate("CX", (a, b)), Gate("RZ", (b,), tuple(g.params)), Gate("CX", (a, b))]
        else:
            out.append(g)
    return out


def cx_sandwich_circuit(n: int, n_blocks: int, seed: int) -> List[Gate]:
    """Random CX(c, t) . M . CX(c, t) blocks: M mixes diagonal gates on c and t
    (Z, S, T, RZ, P, CZ, CP, RZZ, CRZ in either wire order) with gates on other
    qubits; some blocks carry a non-diagonal gate on c or t (no longer a
    diagonal sandwich) and some stand next to diagonal gates on (c, t)."""
    rng = np.random.default_rng(seed)
    diag1 = ("Z", "S", "T", "RZ", "P")
    diag2 = ("CZ", "CP", "RZZ", "CRZ")
    other = ("H", "RX", "RY", "SX", "U3", "CX", "CRY")
    g: List[Gate] = []

    def rand_gate(kinds, wires):
        k = kinds[int(rng.integers(len(kinds)))]
        w = tuple(int(x) for x in rng.permutation(wires)[:arity(k)])
        return Gate(k, w, tuple(float(x) for x in rng.uniform(-np.pi, np.pi, size=N_PARAMS.get(k, 0))))

    for _ in range(n_blocks):
        c, t = (int(x) for x in rng.choice(n, size=2, replace=False))
        rest = [q for q in range(n) if q not in (c, t)]
        if rng.random() < 0.5:
            g.append(rand_gate(diag1, [c, t]))
        g.append(Gate("CX", (c, t)))
        for _ in range(int(rng.integers(0, 5))):
            r = rng.random()
            if r < 0.35:
                g.append(rand_gate(diag1, [c, t]))
            elif r < 0.6:
                g.append(rand_gate(diag2, [c, t]))
            elif r < 0.9 and len(rest) >= 2:
                g.append(rand_gate(other, rest))
            elif r >= 0.9:
                g.append(rand_gate(("H", "RX"), [c, t]))
        g.append(Gate("CX", (c, t)))
        if rng.random() < 0.5:
            g.append(rand_gate(diag1 + diag2, [c, t]))
    return g
