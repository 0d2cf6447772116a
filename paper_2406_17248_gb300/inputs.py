"""Seeded synthetic workloads for the state-vector VQA hot path.

This module only *describes* inputs: gate lists, Pauli-sum Hamiltonians, graphs
and parameter vectors drawn from seeded numpy generators.  It contains none of
the simulation arithmetic (no gate matrices, no amplitudes, no expectations), so
both the FP64 oracle and the CUDA path can consume the same inputs without
sharing any of the method's code.

Workload recipes (shapes follow the paper's benchmarks, §7.1 random circuits and
§7.2 QAOA MaxCut, and the ansatz/Hamiltonian families of §4.2 and §5.2):

* ``random_circuit``   gate kind uniform over {H, RX, RY, RZ, CNOT, CZ}; one-qubit
                       targets uniform in [0, n); two-qubit (control, target)
                       uniform over ordered distinct pairs; angles U[-pi, pi].
* ``hea_circuit``      hardware-efficient ansatz: per layer RY then RZ on every
                       qubit (one parameter each; order layer, qubit, (RY, RZ)),
                       then an open CNOT ladder i -> i+1.
* ``chain_zz_x``       H = sum_i Z_i Z_{i+1} + hx * sum_i X_i on an open chain.
* ``tfim``             H = sum_i J_i Z_i Z_{i+1} + h sum_i X_i, J_i ~ N(1, 0.2),
                       h ~ U[0.5, 1.5].
* ``random_regular_graph``  configuration (pairing) model with rejection of
                       self-loops and multi-edges.
* ``erdos_renyi``      G(n, p).
* ``qaoa_circuit``     |+>^n, then per layer RZZ(gamma_l) on every edge followed by
                       RX(beta_l) on every qubit (cost first, mixer second, §5.2).
* ``lfim``             H_prob = -J sum_i Z_i Z_{i+1} - h sum_i Z_i + k sum_i X_i on an
                       open chain (§5.4; the longitudinal-field case is J = h = 1, k = 0).
* ``dcqaoa_circuit``   DC-QAOA (§5.4): |+>^n, then per layer U_p(gamma_l) =
                       exp(-i gamma_l H_prob), U_m(beta_l) = exp(-i beta_l sum X),
                       U_cd(alpha_l) = exp(-i alpha_l sum Y) with the CD pool term
                       A* = sum_i Y_i.  Parameters per layer (gamma_l, beta_l, alpha_l).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import math

import numpy as np

# Gate kinds understood by both sides (names follow §2.3; CNOT = X with one
# control, CZ = Z with one control, §2.3.5).
FIXED_GATES = ("I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "SWAP")
PARAM_GATES = ("RX", "RY", "RZ", "PS", "RXX", "RYY", "RZZ")
MATRIX_GATES = ("MATRIX",)
ALL_GATES = FIXED_GATES + PARAM_GATES + MATRIX_GATES
TWO_TARGET = ("SWAP", "RXX", "RYY", "RZZ")


@dataclasses.dataclass(frozen=True)
class Gate:
    """One gate record: kind, target qubits, control qubits and its angle binding.

    angle = const + coef * params[param]   (param = -1: fixed angle = const)
    ``matrix`` (row-major, complex) is only used by kind "MATRIX"; its basis index
    is sum_j bit(targets[j]) << j.
    """

    kind: str
    targets: Tuple[int, ...]
    ctrls: Tuple[int, ...] = ()
    param: int = -1
    coef: float = 1.0
    const: float = 0.0
    matrix: Optional[Tuple[complex, ...]] = None

    def angle(self, params: Sequence[float]) -> float:
        if self.param < 0:
            return float(self.const)
        return float(self.const + self.coef * params[self.param])


@dataclasses.dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    n_params: int = 0


@dataclasses.dataclass
class PauliSum:
    """sum_k coef_k * P_k with each P_k given as (xmask, zmask); Y = both bits set."""

    n_qubits: int
    xmask: np.ndarray  # uint64[n_terms]
    zmask: np.ndarray  # uint64[n_terms]
    coef: np.ndarray  # float64[n_terms]

    @property
    def n_terms(self) -> int:
        return int(self.coef.shape[0])


def pauli_sum_from_strings(n_qubits: int, terms: Sequence[Tuple[float, str]]) -> PauliSum:
    """Parse terms like (2.0, "X0 Z1") into masks (§2.5.1 string notation)."""
    xs, zs, cs = [], [], []
    for coef, word in terms:
        x = z = 0
        for tok in word.split():
            p, q = tok[0].upper(), int(tok[1:])
            if not 0 <= q < n_qubits:
                raise ValueError(f"qubit {q} out of range in {word!r}")
            bit = 1 << q
            if (x | z) & bit:
                raise ValueError(f"qubit {q} repeated in {word!r}")
            if p == "X":
                x |= bit
            elif p == "Y":
                x |= bit
                z |= bit
            elif p == "Z":
                z |= bit
            else:
                raise ValueError(f"bad Pauli {p!r}")
        xs.append(x)
        zs.append(z)
        cs.append(float(coef))
    return PauliSum(n_qubits, np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64),
                    np.array(cs, dtype=np.float64))


# --------------------------------------------------------------------------- circuits

def random_circuit(n: int, n_gates: int, seed: int) -> Circuit:
    rng = np.random.default_rng(seed)
    kinds = ("H", "RX", "RY", "RZ", "CNOT", "CZ")
    gates: List[Gate] = []
    for _ in range(n_gates):
        k = kinds[int(rng.integers(0, len(kinds)))]
        if k in ("CNOT", "CZ"):
            c = int(rng.integers(0, n))
            t = int(rng.integers(0, n - 1))
            if t >= c:
                t += 1
            gates.append(Gate("X" if k == "CNOT" else "Z", (t,), (c,)))
        else:
            t = int(rng.integers(0, n))
            if k == "H":
                gates.append(Gate("H", (t,)))
            else:
                gates.append(Gate(k, (t,), const=float(rng.uniform(-np.pi, np.pi))))
    return Circuit(n, gates, 0)


def hea_circuit(n: int, layers: int) -> Circuit:
    gates: List[Gate] = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("RY", (q,), param=p))
            gates.append(Gate("RZ", (q,), param=p + 1))
            p += 2
        for q in range(n - 1):
            gates.append(Gate("X", (q + 1,), (q,)))
    return Circuit(n, gates, p)


def uniform_params(count: int, seed: int, lo: float = -np.pi, hi: float = np.pi) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=count)


def chain_zz_x(n: int, hx: float = 0.5) -> PauliSum:
    terms = [(1.0, f"Z{i} Z{i + 1}") for i in range(n - 1)]
    terms += [(hx, f"X{i}") for i in range(n)]
    return pauli_sum_from_strings(n, terms)


def tfim(n: int, rng: np.random.Generator) -> PauliSum:
    J = rng.normal(1.0, 0.2, size=n - 1)
    h = float(rng.uniform(0.5, 1.5))
    terms = [(float(J[i]), f"Z{i} Z{i + 1}") for i in range(n - 1)]
    terms += [(h, f"X{i}") for i in range(n)]
    return pauli_sum_from_strings(n, terms)


# --------------------------------------------------------------------------- graphs

def random_regular_graph(n: int, d: int, seed: int, max_tries: int = 10000) -> List[Tuple[int, int]]:
    if (n * d) % 2 or d >= n:
        raise ValueError("n*d must be even and d < n")
    rng = np.random.default_rng(seed)
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), d)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        ok = True
        seen = set()
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in seen:
                ok = False
                break
            seen.add(e)
        if ok:
            return sorted(seen)
    raise RuntimeError("pairing model failed")


def erdos_renyi(n: int, p: float, seed: int) -> List[Tuple[int, int]]:
    rng = np.random.default_rng(seed)
    edges = []
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                edges.append((i, j))
    return edges


def complete_graph(n: int) -> List[Tuple[int, int]]:
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def maxcut_zz(n: int, edges: Sequence[Tuple[int, int]]) -> PauliSum:
    return pauli_sum_from_strings(n, [(1.0, f"Z{a} Z{b}") for a, b in edges])


def qaoa_circuit(n: int, edges: Sequence[Tuple[int, int]], p: int, gamma_coef: float = 1.0) -> Circuit:
    """Gate-level QAOA: H on every qubit, then per layer RZZ(gamma_coef*gamma_l) on
    every edge and RX(beta_l) on every qubit.  Parameters: [gamma_1..gamma_p,
    beta_1..beta_p].  gamma_coef = 2 gives the exp(-i gamma sum ZZ) form."""
    gates: List[Gate] = [Gate("H", (q,)) for q in range(n)]
    for l in range(p):
        for a, b in edges:
            gates.append(Gate("RZZ", (a, b), param=l, coef=gamma_coef))
        for q in range(n):
            gates.append(Gate("RX", (q,), param=p + l))
    return Circuit(n, gates, 2 * p)


def lfim(n: int, J: float = 1.0, h: float = 1.0, k: float = 0.0) -> PauliSum:
    """The Ising problem Hamiltonian of the DC-QAOA example (§5.4) on an open chain."""
    terms = [(-J, f"Z{i} Z{i + 1}") for i in range(n - 1)]
    terms += [(-h, f"Z{i}") for i in range(n)]
    if k != 0.0:
        terms += [(k, f"X{i}") for i in range(n)]
    return pauli_sum_from_strings(n, terms)


def dcqaoa_circuit(n: int, p: int, J: float = 1.0, h: float = 1.0, k: float = 0.0, cd: bool = True) -> Circuit:
    """Gate-level DC-QAOA ansatz (§5.4): H on every qubit, then per layer l
    exp(-i gamma_l H_prob) as RZZ(-2 J gamma_l) on each chain bond, RZ(-2 h gamma_l)
    and (k != 0) RX(2 k gamma_l) on each qubit -- exact for k = 0, where the terms
    commute, and the first-order product of the term exponentials otherwise --
    then RX(2 beta_l) on every qubit (mixer sum X) and, with ``cd``, RY(2 alpha_l)
    on every qubit (the counterdiabatic term sum Y).  Parameters, layer by layer:
    (gamma_l, beta_l, alpha_l), or (gamma_l, beta_l) without ``cd``."""
    per = 3 if cd else 2
    gates: List[Gate] = [Gate("H", (q,)) for q in range(n)]
    for l in range(p):
        g, b, a = per * l, per * l + 1, per * l + 2
        for i in range(n - 1):
            gates.append(Gate("RZZ", (i, i + 1), param=g, coef=-2.0 * J))
        for q in range(n):
            gates.append(Gate("RZ", (q,), param=g, coef=-2.0 * h))
        if k != 0.0:
            for q in range(n):
                gates.append(Gate("RX", (q,), param=g, coef=2.0 * k))
        for q in range(n):
            gates.append(Gate("RX", (q,), param=b, coef=2.0))
        if cd:
            for q in range(n):
                gates.append(Gate("RY", (q,), param=a, coef=2.0))
    return Circuit(n, gates, per * p)


# --------------------------------------------------------------------------- batches

@dataclasses.dataclass
class Instance:
    circuit: Circuit
    ham: PauliSum
    params: np.ndarray


def batched_vqe(count: int, seed: int, n_range=(10, 20), depth_range=(2, 10)) -> List[Instance]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        circ = hea_circuit(n, depth)
        ham = tfim(n, rng)
        params = rng.uniform(-np.pi, np.pi, size=circ.n_params)
        out.append(Instance(circ, ham, params))
    return out


# --------------------------------------------------------------------------- test mixes

ONE_Q_KINDS = ("I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "PS")
TWO_Q_KINDS = ("SWAP", "RXX", "RYY", "RZZ")


def random_mixed_circuit(n: int, n_gates: int, seed: int, max_ctrls: int = 2, with_matrix: bool = True) -> Circuit:
    """Every gate kind, random targets and 0..max_ctrls controls, linear angle
    bindings (own parameter per rotation), optionally one random 2-qubit unitary.
    The unitary is drawn as the Q factor of a complex Gaussian matrix."""
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    p = 0
    for _ in range(n_gates):
        two = rng.random() < 0.3 and n >= 2
        kinds = TWO_Q_KINDS if two else ONE_Q_KINDS
        kind = kinds[int(rng.integers(len(kinds)))]
        qs = [int(q) for q in rng.permutation(n)]
        nt = 2 if two else 1
        targets = tuple(qs[:nt])
        nc = int(rng.integers(0, min(max_ctrls, n - nt) + 1))
        ctrls = tuple(qs[nt:nt + nc])
        if kind in PARAM_GATES:
            gates.append(Gate(kind, targets, ctrls, param=p, coef=float(rng.uniform(-2, 2)),
                              const=float(rng.uniform(-1, 1))))
            p += 1
        else:
            gates.append(Gate(kind, targets, ctrls))
    if with_matrix and n >= 2 and rng.random() < 0.5:
        a = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
        q, _ = np.linalg.qr(a)
        gates.append(Gate("MATRIX", (1, 0), (), matrix=tuple(complex(v) for v in q.reshape(-1))))
    return Circuit(n, gates, p)


def random_pauli_sum(n: int, n_terms: int, seed: int) -> PauliSum:
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(n_terms):
        word = " ".join(f"{'XYZ'[int(rng.integers(3))]}{q}" for q in range(n) if rng.random() < 0.5)
        terms.append((float(rng.normal()), word))
    return pauli_sum_from_strings(n, terms)


def random_state(n: int, seed: int) -> np.ndarray:
    """A normalised complex Gaussian vector (an input state, not a simulation result)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------------- graph sets (learned QAOA initialiser)

def graph_set(count: int, seed: int, n_range=(16, 26), er_p: float = 0.3) -> List[Tuple[int, List[Tuple[int, int]]]]:
    """`count` graphs: even positions random 3-regular (pairing model), odd
    positions Erdos-Renyi G(n, er_p); n ~ U{n_range} (3-regular graphs take the
    next even n when n is odd).  Returns [(n, edges)]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        s = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            if n % 2:
                n = n + 1 if n + 1 <= n_range[1] else n - 1
            out.append((n, random_regular_graph(n, 3, s)))
        else:
            out.append((n, erdos_renyi(n, er_p, s)))
    return out


def pack_graphs(graphs: Sequence[Tuple[int, Sequence[Tuple[int, int]]]]):
    """CSR batch of undirected graphs: node_off[G+1] (graph g owns global nodes
    node_off[g] .. node_off[g+1]-1), adj_off[N+1] and adj[2E] (neighbours of
    global node v are adj[adj_off[v] .. adj_off[v+1]), as LOCAL indices within
    v's graph, in increasing order).  int32 numpy arrays."""
    node_off = [0]
    adj_off = [0]
    adj: List[int] = []
    for n, edges in graphs:
        nb: List[List[int]] = [[] for _ in range(n)]
        for a, b in edges:
            nb[a].append(b)
            nb[b].append(a)
        for v in range(n):
            adj.extend(sorted(nb[v]))
            adj_off.append(len(adj))
        node_off.append(node_off[-1] + n)
    return (np.array(node_off, dtype=np.int32), np.array(adj_off, dtype=np.int32),
            np.array(adj if adj else [0], dtype=np.int32)[: len(adj)])


def gnn_init_weights(n_weights_layout, seed: int) -> np.ndarray:
    """Glorot-uniform weights and zero biases for a flat parameter vector
    described by [(kind, rows, cols)] blocks ('W' or 'b'), float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for kind, rows, cols in n_weights_layout:
        if kind == "W":
            lim = np.sqrt(6.0 / (rows + cols))
            parts.append(rng.uniform(-lim, lim, size=rows * cols))
        else:
            parts.append(np.zeros(rows))
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------- large states by formula

def hashed_amplitudes(idx: np.ndarray, seed: int, n: int) -> np.ndarray:
    """Amplitudes of a seeded pseudo-random state given index by index, so that
    states too large to hold on the host can be generated in chunks and any
    amplitude recomputed: a_x = (u - 1/2 + i (v - 1/2)) * 2^{(1 - n)/2} * sqrt(3),
    u, v the top 53 bits of two splitmix64 outputs of the counter (seed, x).
    The squared norm is close to 1 (the mean of |a_x|^2 is 2^-n)."""
    x = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        def mix(z):
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            return z ^ (z >> np.uint64(31))
        g = np.uint64(0x9E3779B97F4A7C15)
        base = np.uint64(seed) * np.uint64(0xD1B54A32D192ED03) + x * np.uint64(2) * g
        u = (mix(base + g) >> np.uint64(11)).astype(np.float64) * 2.0**-53
        v = (mix(base + g + g) >> np.uint64(11)).astype(np.float64) * 2.0**-53
    s = math.sqrt(3.0) * 2.0 ** ((1 - n) / 2)
    return ((u - 0.5) + 1j * (v - 0.5)) * s
