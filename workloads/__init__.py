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


# ----------------------------------------------------------------------------
# the end-to-end workload sweep (App. sweep table: every gate-based family of
# the paper's suite).  The paper names the families; the circuits below are
# this package's own seeded readings of them (sizes, step counts, angles).
# ----------------------------------------------------------------------------
def long_range_ising_gates(n: int, steps: int, dt: float, J: float = 1.0, h: float = 0.5,
                           alpha: float = 1.5) -> List[Gate]:
    """All-to-all Ising with couplings J / d^alpha over distance d (Sec. 5.1:
    n(n-1)/2 bonds in n-1 equal-angle distance groups), first order: per step
    RZZ(-2 J_d dt) on every pair, then RX(2 h dt) on every qubit."""
    g: List[Gate] = []
    for _ in range(steps):
        for i in range(n):
            for j in range(i + 1, n):
                g.append(Gate("RZZ", (i, j), (-2.0 * J * dt / float(j - i) ** alpha,)))
        g += [Gate("RX", (q,), (2.0 * h * dt,)) for q in range(n)]
    return g


def heisenberg_gates(n: int, steps: int, dt: float, J: float = 1.0, delta: float = 1.0,
                     fields=None) -> List[Gate]:
    """H = J sum_i (X_i X_{i+1} + Y_i Y_{i+1} + delta Z_i Z_{i+1}) (+ sum_i h_i Z_i)
    on an open chain, first order: per step the XX terms on every bond, then
    the YY terms, then the ZZ terms (same-family runs, Sec. 5.1), then RZ(2 h_i dt)."""
    g: List[Gate] = []
    for _ in range(steps):
        g += [Gate("RXX", (b, b + 1), (2.0 * J * dt,)) for b in range(n - 1)]
        g += [Gate("RYY", (b, b + 1), (2.0 * J * dt,)) for b in range(n - 1)]
        g += [Gate("RZZ", (b, b + 1), (2.0 * J * delta * dt,)) for b in range(n - 1)]
        if fields is not None:
            g += [Gate("RZ", (q,), (2.0 * float(fields[q]) * dt,)) for q in range(n)]
    return g


def heisenberg_ladder_gates(n: int, steps: int, dt: float, J: float = 1.0) -> List[Gate]:
    """Two-leg ladder (legs q and q + n/2, rungs between them), first order with
    the XX, YY and ZZ terms of each bond in turn (no same-family run exists)."""
    half = n // 2
    bonds = [(q, q + 1) for q in range(half - 1)] + [(q, q + 1) for q in range(half, n - 1)]
    bonds += [(q, q + half) for q in range(half)]
    g: List[Gate] = []
    for _ in range(steps):
        for a, b in bonds:
            g += [Gate("RXX", (a, b), (2.0 * J * dt,)), Gate("RYY", (a, b), (2.0 * J * dt,)),
                  Gate("RZZ", (a, b), (2.0 * J * dt,))]
    return g


def rotation_entangler_gates(n: int, layers: int, seed: int, rot=("RY", "RZ"), ent: str = "CX",
                             final: bool = True) -> List[Gate]:
    """Hardware-efficient layers: the rotations `rot` on every qubit with angles
    ~ U[0, 2 pi), then `ent` on (q, q+1) for q = 0..n-2; a last rotation layer
    when `final` (EfficientSU2: RY RZ + CX; RealAmplitudes: RY + CX; QCBM:
    RX RZ + CX; QNN layer: RY + CZ)."""
    rng = np.random.default_rng(seed)
    g: List[Gate] = []
    for _ in range(layers):
        for r in rot:
            g += [Gate(r, (q,), (float(rng.uniform(0, 2 * np.pi)),)) for q in range(n)]
        g += [Gate(ent, (q, q + 1)) for q in range(n - 1)]
    if final:
        for r in rot:
            g += [Gate(r, (q,), (float(rng.uniform(0, 2 * np.pi)),)) for q in range(n)]
    return g


def graph_state_gates(n: int, seed: int, chords: int = 0) -> List[Gate]:
    """H on every qubit, then CZ on the ring edges and `chords` random extra edges."""
    rng = np.random.default_rng(seed)
    edges = [(q, (q + 1) % n) for q in range(n)]
    while len(edges) < n + chords:
        u, v = (int(x) for x in rng.choice(n, size=2, replace=False))
        if (u, v) not in edges and (v, u) not in edges:
            edges.append((u, v))
    return [Gate("H", (q,)) for q in range(n)] + [Gate("CZ", e) for e in edges]


def qpe_gates(n: int, phi: float) -> List[Gate]:
    """Phase estimation of U = P(phi) on qubit n-1 (eigenstate |1>, prepared by
    X) with counting qubits 0..n-2: H on each, CP(phi 2^k) from counting qubit
    n-2-k to the target (the controlled-power ladder, angles up to
    phi 2^(n-2)), then the inverse QFT on the counting register (the QFT's
    gates in reverse order with negated angles)."""
    m = n - 1
    g: List[Gate] = [Gate("X", (n - 1,))] + [Gate("H", (q,)) for q in range(m)]
    for k in range(m):
        g.append(Gate("CP", (m - 1 - k, n - 1), (phi * float(2 ** k),)))
    inv = []
    for gt in reversed(qft_gates(m, swaps=True)):
        inv.append(Gate(gt.kind, gt.wires, tuple(-p for p in gt.params)))
    return g + inv


def qpe_exact_phase(n: int, seed: int) -> float:
    """A phase 2 pi j / 2^(n-1) that n-1 counting qubits resolve exactly (j seeded)."""
    m = n - 1
    j = int(np.random.default_rng(seed).integers(1, 2 ** m))
    return 2.0 * np.pi * j / float(2 ** m)


def deutsch_jozsa_gates(n: int, seed: int) -> List[Gate]:
    """Inputs 0..n-2, ancilla n-1: X and H on the ancilla, H on the inputs, a
    balanced oracle (CX from the inputs in a random nonzero mask to the
    ancilla, X on a random subset of inputs around it), H on the inputs."""
    rng = np.random.default_rng(seed)
    m = n - 1
    mask = [q for q in range(m) if rng.random() < 0.5] or [0]
    flip = [q for q in range(m) if rng.random() < 0.3]
    g = [Gate("X", (m,)), Gate("H", (m,))] + [Gate("H", (q,)) for q in range(m)]
    g += [Gate("X", (q,)) for q in flip]
    g += [Gate("CX", (q, m)) for q in mask]
    g += [Gate("X", (q,)) for q in flip]
    return g + [Gate("H", (q,)) for q in range(m)]


def w_state_gates(n: int) -> List[Gate]:
    """W state by the controlled-rotation cascade: X on qubit 0, then for
    k = 0..n-2: CRY(2 arccos sqrt(1 / (n - k))) from k to k+1, CX(k+1, k)."""
    g = [Gate("X", (0,))]
    for k in range(n - 1):
        g.append(Gate("CRY", (k, k + 1), (2.0 * float(np.arccos(np.sqrt(1.0 / (n - k)))),)))
        g.append(Gate("CX", (k + 1, k)))
    return g


def amplitude_estimation_gates(n: int, rounds: int, seed: int) -> List[Gate]:
    """Single CZ gates between short single-qubit blocks (the structure the
    paper's amplitude-estimation row has): per round and qubit q, RY and H on
    q, then CZ(q, q+1)."""
    rng = np.random.default_rng(seed)
    g: List[Gate] = []
    for _ in range(rounds):
        for q in range(n - 1):
            g += [Gate("RY", (q,), (float(rng.uniform(0, np.pi)),)), Gate("H", (q,)), Gate("CZ", (q, q + 1))]
    return g


def grover_vchain_gates(n: int, marked: int, iterations: int) -> List[Gate]:
    """Grover search on m = (n + 3) // 2 data qubits (0..m-1) with m - 3
    ancillas (m..2m-4) for the multi-controlled Z, built from CCX as a V-chain:
    the ancillas collect the AND of the controls, CCX onto the last data
    qubit between H gates flips the phase, and the chain is undone, leaving the
    ancillas in |0>.  Start H on the data; per iteration: the oracle (X on the
    data qubits where `marked`, read with qubit 0 as its most significant
    bit, is 0, then MCZ, then the X again) and the diffusion H X MCZ X H."""
    m = (n + 3) // 2
    if m < 3 or 2 * m - 3 > n:
        raise ValueError("grover_vchain_gates needs n >= 3")
    data = list(range(m))
    anc = list(range(m, 2 * m - 3))

    def mcz():
        c, t = data[:-1], data[-1]
        chain: List[Gate] = []
        if len(c) == 2:
            core = [Gate("CCX", (c[0], c[1], t))]
        else:
            chain.append(Gate("CCX", (c[0], c[1], anc[0])))
            for i in range(2, len(c) - 1):
                chain.append(Gate("CCX", (c[i], anc[i - 2], anc[i - 1])))
            core = [Gate("CCX", (c[-1], anc[len(c) - 3], t))]
        return [Gate("H", (t,))] + chain + core + list(reversed(chain)) + [Gate("H", (t,))]

    zeros = [q for q in data if not (marked >> (m - 1 - q)) & 1]
    g: List[Gate] = [Gate("H", (q,)) for q in data]
    for _ in range(iterations):
        g += [Gate("X", (q,)) for q in zeros] + mcz() + [Gate("X", (q,)) for q in zeros]
        g += [Gate("H", (q,)) for q in data] + [Gate("X", (q,)) for q in data] + mcz()
        g += [Gate("X", (q,)) for q in data] + [Gate("H", (q,)) for q in data]
    return g


def quantum_walk_gates(n: int, steps: int) -> List[Gate]:
    """Coined walk on a cycle of 2^p positions, p = n // 2: coin qubit 0,
    position bits r_j = qubit 1 + j (r_0 least significant), p - 1 ancillas
    after them.  One step: H on the coin, then position + 1 where the coin is
    1 and position - 1 where it is 0 (mod 2^p).  The increment is the carry
    chain: the ancillas collect coin AND r_0 AND ... AND r_j (CCX V-chain), each
    r_{j+1} flips by CX from the chain, highest first, while the chain is
    undone, and r_0 flips by CX from the coin; the decrement is the increment
    between X layers on the position and the coin."""
    p = n // 2
    if p < 2:
        raise ValueError("quantum_walk_gates needs n >= 4")
    coin, r = 0, [1 + j for j in range(p)]
    a = [1 + p + j for j in range(p - 1)]

    def increment() -> List[Gate]:
        g = [Gate("CCX", (coin, r[0], a[0]))]
        for j in range(1, p - 1):
            g.append(Gate("CCX", (a[j - 1], r[j], a[j])))
        for j in range(p - 2, -1, -1):
            g.append(Gate("CX", (a[j], r[j + 1])))
            g.append(Gate("CCX", (a[j - 1], r[j], a[j])) if j > 0 else Gate("CCX", (coin, r[0], a[0])))
        g.append(Gate("CX", (coin, r[0])))
        return g

    g: List[Gate] = []
    for _ in range(steps):
        g.append(Gate("H", (coin,)))
        g += increment()
        flip = [Gate("X", (q,)) for q in [coin] + r]
        g += flip + increment() + flip
    return g


def sweep_workloads(n: int, seed: int = 11):
    """The sweep's gate-based families at n qubits: (name, gates)."""
    rng = np.random.default_rng(seed)
    f = tfim_fields(n, seed)
    out = [
        ("tfim_2nd_order", tfim_gates(n, 20, 0.05, 1.0, f, order=2)),
        ("tfim_1st_order", tfim_gates(n, 20, 0.05, 1.0, 0.5, order=1)),
        ("tfim_random_field", tfim_gates(n, 20, 0.05, 1.0, rng.uniform(0.0, 2.0, size=n), order=1)),
        ("long_range_ising", long_range_ising_gates(n, 4, 0.05)),
        ("heisenberg_chain", heisenberg_gates(n, 10, 0.05)),
        ("heisenberg_xxz", heisenberg_gates(n, 10, 0.05, delta=0.5)),
        ("heisenberg_random_field", heisenberg_gates(n, 10, 0.05, fields=rng.uniform(-1, 1, size=n))),
        ("heisenberg_2leg_ladder", heisenberg_ladder_gates(n, 4, 0.05)),
        ("variational_ansatz", [Gate(x.kind, x.wires, x.params) for x in
                                bind_params(vqe_ansatz_gates(n, 6), vqe_params(n, 6, 1, seed)[0])]),
        ("efficient_su2", rotation_entangler_gates(n, 4, seed, ("RY", "RZ"), "CX")),
        ("real_amplitudes", rotation_entangler_gates(n, 4, seed + 1, ("RY",), "CX")),
        ("qcbm", rotation_entangler_gates(n, 9, seed + 2, ("RX", "RZ"), "CX", final=False)),
        ("qnn_layer", rotation_entangler_gates(n, 2, seed + 3, ("RY",), "CZ")),
        ("ghz", ghz_gates(n)),
        ("graph_state", graph_state_gates(n, seed, chords=n // 2)),
        ("qft", qft_gates(n, swaps=True)),
        ("qft_entangled_input", ghz_gates(n) + qft_gates(n, swaps=True)),
        ("phase_estimation", qpe_gates(n, qpe_exact_phase(n, seed))),
        ("phase_estimation_inexact", qpe_gates(n, 0.4)),   # ladder angles up to 0.4 * 2^(n-2) rad
        ("qaoa_ring", qaoa_gates(n, [(q, (q + 1) % n) for q in range(n)], [0.4, 0.8, 1.1, 0.3],
                                 [0.7, 0.5, 0.2, 0.9])),
        ("deutsch_jozsa", deutsch_jozsa_gates(n, seed)),
        ("random_circuit", random_circuit(n, 10 * n, seed, [k for k in ONE_QUBIT + TWO_QUBIT + THREE_QUBIT
                                                             if k != "U"])),
        ("amplitude_estimation", amplitude_estimation_gates(n, 3, seed)),
        ("w_state", w_state_gates(n)),
        ("grover_search", grover_vchain_gates(n, int(rng.integers(1, 2 ** ((n + 3) // 2))), 2)),
        ("quantum_walk", quantum_walk_gates(n, 4)),
    ]
    return out
