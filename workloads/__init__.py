"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only *describes* circuits and draws the random numbers that are
inputs of the method (basis states, marked indices, Haar-random gate matrices,
ansatz angles).  It holds none of the method's arithmetic: it never applies a
gate, never builds a matrix from an angle and never touches a state vector.
Both the CUDA library binding and the CPU oracle translate these descriptions
into their own gate structures.

Conventions of the paper (quant-ph/0201042):
  * qubit 0 is the most significant bit of the amplitude index (Sec. 2.2.1);
  * gate kinds follow the paper's vocabulary: H (Sec. 2.3.1), the rotation U_R
    and the phase shifts U_P1, U_P2 (Sec. 3.2), Pauli X/Y/Z (Sec. 3.1), plus the
    RY/RZ rotations of the variational ansatz and explicit 2x2 matrices.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# Gate kinds and the number of angles each carries.
KINDS = {
    "MATRIX": 0, "H": 0, "X": 0, "Y": 0, "Z": 0,
    "UP1": 1, "UP2": 1, "UR": 1, "URP1": 2, "RY": 1, "RZ": 1, "SWAP": 0,
}


@dataclass
class Gate:
    """One gate of a circuit.

    kind     one of KINDS
    target   target qubit (0 = most significant index bit)
    target2  second qubit of a SWAP, else -1
    controls {qubit: required value (0 or 1)}
    angles   angles of the kind (radians), e.g. (phi,) for UP1, (theta, phi) for URP1
    matrix   2x2 complex matrix for kind MATRIX (row major), else None
    param    index of angles[0] in a parameter vector (differentiable gates), else -1
    """
    kind: str
    target: int
    target2: int = -1
    controls: Dict[int, int] = field(default_factory=dict)
    angles: Tuple[float, ...] = ()
    matrix: Optional[np.ndarray] = None
    param: int = -1

    def ctrl_mask(self) -> int:
        m = 0
        for q in self.controls:
            m |= 1 << q
        return m

    def ctrl_val(self) -> int:
        v = 0
        for q, b in self.controls.items():
            if b:
                v |= 1 << q
        return v


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


# --------------------------------------------------------------------------
# Circuits of the paper and of the workloads built on it
# --------------------------------------------------------------------------

def hadamard_layer(n: int) -> List[Gate]:
    """H on every qubit: the Hadamard transform H_n (Sec. 2.3.1)."""
    return [Gate("H", q) for q in range(n)]


def qft_circuit(n: int, q0: int = 0, L: Optional[int] = None, max_k: Optional[int] = None) -> List[Gate]:
    """The textbook QFT circuit for beta_x = 2^{-L/2} sum_y w^{xy} alpha_y with
    w = e^{2 pi i / 2^L} (Sec. 2.3.2) on the L qubits q0 .. q0+L-1 (q0 the most
    significant; L defaults to n - q0): for each qubit j of the register, H on j
    followed by the phase shifts diag(1, e^{2 pi i / 2^k}) on target j controlled
    by qubit j+k-1, k = 2..; then SWAPs reverse the register's qubit order.  The
    paper's R_d = diag(1, e^{i pi / 2^d}) is the same gate with d = k - 1.

    max_k: the approximate QFT of Sec. 2.3.2 -- phase shifts with k > max_k
    (angles below 2 pi / 2^max_k, which act on distant qubits) are left out."""
    if L is None:
        L = n - q0
    gates: List[Gate] = []
    for j in range(L):
        gates.append(Gate("H", q0 + j))
        for k in range(2, L - j + 1):
            if max_k is not None and k > max_k:
                break
            gates.append(Gate("UP1", q0 + j, controls={q0 + j + k - 1: 1},
                              angles=(2.0 * math.pi / (1 << k),)))
    for j in range(L // 2):
        gates.append(Gate("SWAP", q0 + j, target2=q0 + L - 1 - j))
    return gates


def approx_qft_max_k(L: int, eps: float) -> int:
    """Largest phase-shift index k kept by the approximate QFT of accuracy eps
    (Sec. 2.3.2: O(L log(L / eps)) gates): k <= ceil(log2(L / eps)), at least 2."""
    return max(2, int(math.ceil(math.log2(L / eps))))


def phase_flip(n: int, index: int, phi: float = math.pi) -> Gate:
    """Phase e^{i phi} on the single amplitude `index` (phi = pi: the sign
    changing operator V_f of Grover's iteration, Sec. 5.3): a phase shift on
    the least significant qubit, controlled by every other qubit."""
    t = n - 1
    controls = {q: (index >> (n - 1 - q)) & 1 for q in range(n - 1)}
    kind = "UP1" if index & 1 else "UP2"
    return Gate(kind, t, controls=controls, angles=(phi,))


def grover_circuit(n: int, marked: int, iters: int) -> List[Gate]:
    """H_n, then `iters` G-iterations  V_{f_k}, H_n, V_{f_0}, H_n  (Sec. 5.3,
    G = -H_n V_{f_0} H_n V_{f_k}).  The global factor -1 of G is left out: the
    state after j iterations is (-1)^j times the closed form."""
    gates = hadamard_layer(n)
    for _ in range(iters):
        gates.append(phase_flip(n, marked))
        gates += hadamard_layer(n)
        gates.append(phase_flip(n, 0))
        gates += hadamard_layer(n)
    return gates


def grover_iterations(n: int) -> int:
    return int(math.floor(math.pi / 4.0 * math.sqrt(2.0 ** n)))


def haar_su2(r: np.random.Generator) -> np.ndarray:
    """Haar-random SU(2) element [[a, -conj(b)], [b, conj(a)]] with (a, b) a
    uniform point of the unit sphere S^3 (4 normalised Gaussians)."""
    v = r.standard_normal(4)
    v = v / np.sqrt(np.sum(v * v))
    a = complex(v[0], v[1])
    b = complex(v[2], v[3])
    return np.array([[a, -b.conjugate()], [b, a.conjugate()]], dtype=np.complex128)


def random_circuit(n: int, layers: int, seed: int) -> List[Gate]:
    """`layers` layers of Haar-random SU(2) gates on every qubit followed by
    CNOTs on n//2 disjoint random (control, target) pairs."""
    r = rng(seed)
    gates: List[Gate] = []
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("MATRIX", q, matrix=haar_su2(r)))
        perm = r.permutation(n)
        for k in range(n // 2):
            c, t = int(perm[2 * k]), int(perm[2 * k + 1])
            gates.append(Gate("X", t, controls={c: 1}))
    return gates


def ansatz_circuit(n: int, layers: int, seed: int) -> Tuple[List[Gate], np.ndarray]:
    """Variational ansatz: per layer RY(theta) on every qubit, RZ(phi) on every
    qubit, then CNOT(q, q+1) for q = 0..n-2.  Angles uniform in [-pi, pi).
    Returns the gates (each rotation carries its parameter index) and the
    parameter vector."""
    r = rng(seed)
    n_par = layers * 2 * n
    params = r.uniform(-math.pi, math.pi, size=n_par)
    gates: List[Gate] = []
    k = 0
    for _ in range(layers):
        for kind in ("RY", "RZ"):
            for q in range(n):
                gates.append(Gate(kind, q, angles=(float(params[k]),), param=k))
                k += 1
        for q in range(n - 1):
            gates.append(Gate("X", q + 1, controls={q: 1}))
    return gates, params


def noisy_synthesis(gates: Sequence[Gate]) -> List[Gate]:
    """Rewrites H, X (with its controls) and Z-type phases in the paper's
    rotation/phase-shift synthesis so that operational errors can deviate their
    angles (Sec. 3.2): H = U_R(pi/4) U_P1(pi), NOT = U_R(pi/2) U_P1(pi),
    Z = U_P1(pi).  Other gates are kept."""
    out: List[Gate] = []
    for g in gates:
        if g.kind == "H":
            out.append(Gate("URP1", g.target, controls=dict(g.controls),
                            angles=(math.pi / 4, math.pi)))
        elif g.kind == "X":
            out.append(Gate("URP1", g.target, controls=dict(g.controls),
                            angles=(math.pi / 2, math.pi)))
        elif g.kind == "Z":
            out.append(Gate("UP1", g.target, controls=dict(g.controls), angles=(math.pi,)))
        else:
            out.append(g)
    return out


NO_DEVIATION = 1   # trajectory gate flag: angles not deviated
NO_FLIPS = 2       # trajectory gate flag: no flips after the gate


def period_finding_qft(n: int, r_log2: int, offset: int, approx_max_k: Optional[int] = None
                       ) -> Tuple[List[Gate], List[int]]:
    """The QFT step of Shor's algorithm (Sec. 5.1, step 3(d); Sec. 5.2): the
    register holds the periodic superposition sum_j |offset + j 2^r_log2>
    (the first register after the second one was measured, the period a power
    of two), prepared without error, then the QFT circuit in the paper's
    synthesis.  Returns (gates, flags): the preparation (X on the offset bits,
    H on the top n - r_log2 qubits) has no deviation and no flips; in the QFT,
    every angle is deviated and flips follow the controlled phase shifts R_d
    only (Sec. 5.2: decoherence each time R_d is applied)."""
    prep: List[Gate] = []
    for b in range(r_log2):
        if (offset >> b) & 1:
            prep.append(Gate("X", n - 1 - b))
    prep += [Gate("H", q) for q in range(n - r_log2)]
    qft = noisy_synthesis(qft_circuit(n, max_k=approx_max_k))
    flags = [NO_DEVIATION | NO_FLIPS] * len(prep)
    for g in qft:
        flags.append(0 if (g.kind == "UP1" and g.controls) else NO_FLIPS)
    return prep + qft, flags


def basis_index(seed: int, n: int) -> int:
    """A basis state index uniform in [0, 2^n)."""
    return int(rng(seed).integers(0, 1 << n))


# --------------------------------------------------------------------------
# Batched noisy trajectories
# --------------------------------------------------------------------------

@dataclass
class TrajectoryBatch:
    """Trajectories grouped by (width, circuit).  For group g, trajectories
    `first[g] .. first[g] + count[g] - 1` (global trajectory ids, which are
    also the Philox counters) run `circuits[g]` on `widths[g]` qubits from the
    basis states `x0[first[g] + i]`; `kinds[g]` is 'qft' (metric: fidelity to
    the noiseless output) or 'grover' (metric: probability of `marked[g]`)."""
    widths: List[int]
    kinds: List[str]
    circuits: List[List[Gate]]
    marked: List[int]
    first: List[int]
    count: List[int]
    x0: np.ndarray


def trajectory_batch(n_traj: int, widths_ratio: Sequence[Tuple[int, int]],
                     grover_widths: Sequence[int], seed: int,
                     grover_iters: Optional[Dict[int, int]] = None) -> TrajectoryBatch:
    """Mixes widths in the given ratio, e.g. ((12, 2), (16, 1), (20, 1)).  At the
    widths listed in `grover_widths` half of the trajectories run Grover and
    half run the QFT; at the other widths all run the QFT on seeded basis
    states.  Every gate is in the rotation/phase synthesis of Sec. 3.2."""
    r = rng(seed)
    tot = sum(w for _, w in widths_ratio)
    counts = [n_traj * w // tot for _, w in widths_ratio]
    counts[0] += n_traj - sum(counts)
    widths, kinds, circuits, marked, first, count = [], [], [], [], [], []
    x0 = np.zeros(n_traj, dtype=np.uint64)
    nxt = 0
    for (n, _), c in zip(widths_ratio, counts):
        parts = [("qft", c)]
        if n in grover_widths:
            parts = [("qft", c - c // 2), ("grover", c // 2)]
        for kind, cc in parts:
            if cc == 0:
                continue
            if kind == "qft":
                circ = noisy_synthesis(qft_circuit(n))
                mk = -1
                x0[nxt:nxt + cc] = r.integers(0, 1 << n, size=cc, dtype=np.uint64)
            else:
                mk = int(r.integers(0, 1 << n))
                it = (grover_iters or {}).get(n, grover_iterations(n))
                circ = noisy_synthesis(grover_circuit(n, mk, it))
                x0[nxt:nxt + cc] = 0
            widths.append(n); kinds.append(kind); circuits.append(circ)
            marked.append(mk); first.append(nxt); count.append(cc)
            nxt += cc
    return TrajectoryBatch(widths, kinds, circuits, marked, first, count, x0)
