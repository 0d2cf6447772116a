"""FP64 CPU oracle of Monte-Carlo trajectory noise (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm may import this module; the product never calls it and shares no
code with it.

Written from §3.3: besides the density-matrix simulator, the state-vector
simulator treats a quantum channel by the Monte-Carlo method -- each noise gate
acts with some probability, and averaging over many sampled runs of the circuit
gives the noisy result.  For a channel with Kraus operators K_i
(Psi(rho) = sum_i K_i rho K_i^dag) one trajectory replaces psi by
K_i psi / ||K_i psi|| with probability ||K_i psi||^2, so that the average of
|psi><psi| over trajectories is Psi(|psi><psi|).

Conventions fixed here (the paper does not print them):

* channel sites are numbered 0, 1, ... in circuit order (the channels attached
  before the first gate, key -1, first; within one gate, list order);
* the uniform of trajectory t at site s is ``shot_uniform(seed, t * n_sites + s)``
  -- splitmix64 (Steele, Lea & Flood 2014) of the counter, top 53 bits;
* branch weights: for the Pauli channel (px, py, pz) the fixed probabilities
  w = (max(0, 1 - px - py - pz), px, py, pz) and for the depolarizing channel (p), with
  q = p / 4, w = (1 - q - q - q, q, q, q), each evaluated left to right in FP64;
  the branch operator is then the Pauli itself (I, X, Y, Z), a unitary.  For the
  damping channels and custom Kraus sets, w_i = ||K_i psi||^2 and the branch
  operator is K_i / sqrt(w_i);
* branch choice: the smallest i whose running sum w_0 + ... + w_i exceeds
  u * (w_0 + ... + w_last); if rounding leaves none, the last i with w_i > 0.

Parity: pinned in tests/test_traj_oracle.py -- exact enumeration of every branch
sequence weighted by its probability against the density-matrix oracle
(energies and, for Pauli channels, gradients against finite differences of the
exact noisy energy), zero-probability channels against the noiseless state,
branch frequencies against the channel probabilities.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

from oracle import dm_oracle as D
from oracle import qsim_oracle as O
from paper_2406_17248_gb300.inputs import Circuit, Gate, PauliSum

_PAULI = (np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], dtype=complex),
          np.array([[0, -1j], [1j, 0]], dtype=complex), np.array([[1, 0], [0, -1]], dtype=complex))
_PAULI_NAMES = ("I", "X", "Y", "Z")


def sites(channels_after: Dict[int, list], n_gates: int) -> List[Tuple[int, tuple]]:
    """[(gate index the site follows, (kind, p, qubit[, kraus]))] in site order."""
    out = []
    for key in [-1] + list(range(n_gates)):
        for ch in channels_after.get(key, []):
            out.append((key, ch))
    return out


def fixed_weights(kind: str, p: Sequence[float]):
    """Branch probabilities of a mixture-of-Paulis channel, or None."""
    if kind == "pauli":
        px, py, pz = (float(v) for v in p)
        return [max(0.0, 1.0 - px - py - pz), px, py, pz]
    if kind == "depolarizing":
        q = float(p[0]) / 4.0
        return [1.0 - q - q - q, q, q, q]
    return None


def kraus_of(ch) -> List[np.ndarray]:
    kind, p = ch[0], ch[1]
    if kind == "kraus":
        return [np.asarray(k, dtype=complex).reshape(2, 2) for k in ch[3]]
    return D.channel_kraus(kind, p)


def choose(w: Sequence[float], u: float) -> int:
    total = 0.0
    for x in w:
        total += x
    thr = u * total
    cum = 0.0
    for i, x in enumerate(w):
        cum += x
        if cum > thr:
            return i
    return max(i for i, x in enumerate(w) if x > 0)


def branch_operator(ch, psi: np.ndarray, n: int, i: int, w: Sequence[float]) -> np.ndarray:
    if fixed_weights(ch[0], ch[1]) is not None:
        return _PAULI[i]
    return kraus_of(ch)[i] / math.sqrt(w[i])


def branch_weights(ch, psi: np.ndarray, n: int) -> List[float]:
    fw = fixed_weights(ch[0], ch[1])
    if fw is not None:
        return fw
    q = ch[2]
    return [float(np.sum(np.abs(O.apply_gate(psi, n, K, [q])) ** 2)) for K in kraus_of(ch)]


def trajectory(circ: Circuit, params, channels_after: Dict[int, list], seed: int, t: int):
    """One trajectory from |0..0>: returns (final state, branch indices, margins),
    margin = distance of u * total from the nearest running sum (how far the
    decision is from flipping under rounding)."""
    n = circ.n_qubits
    st = sites(channels_after, len(circ.gates))
    n_sites = len(st)
    psi = O.zero_state(n)
    choices, margins = [], []
    s = 0

    def do_site(psi, ch):
        nonlocal s
        w = branch_weights(ch, psi, n)
        u = O.shot_uniform(seed, t * n_sites + s)
        i = choose(w, u)
        total = sum(w)
        cums = np.cumsum(w)
        margins.append(float(np.min(np.abs(cums - u * total))))
        choices.append(i)
        s += 1
        return O.apply_gate(psi, n, branch_operator(ch, psi, n, i, w), [ch[2]])

    for ch in channels_after.get(-1, []):
        psi = do_site(psi, ch)
    for gi, g in enumerate(circ.gates):
        psi = O.apply_gate(psi, n, O.gate_unitary(g, params), list(g.targets), list(g.ctrls))
        for ch in channels_after.get(gi, []):
            psi = do_site(psi, ch)
    return psi, choices, margins


def branch_circuit(circ: Circuit, channels_after: Dict[int, list], choices: Sequence[int]) -> Circuit:
    """The unitary circuit of one trajectory of mixture-of-Paulis channels: the
    chosen Pauli inserted at every site (I as an identity gate)."""
    gates: List[Gate] = []
    s = 0
    for ch in channels_after.get(-1, []):
        gates.append(Gate(_PAULI_NAMES[choices[s]], (ch[2],)))
        s += 1
    for gi, g in enumerate(circ.gates):
        gates.append(g)
        for ch in channels_after.get(gi, []):
            gates.append(Gate(_PAULI_NAMES[choices[s]], (ch[2],)))
            s += 1
    return Circuit(circ.n_qubits, gates, circ.n_params)


def trajectory_energy_and_grad(circ: Circuit, ham: PauliSum, params, channels_after, seed: int, t: int):
    """Energy and adjoint gradient of one trajectory (mixture-of-Paulis channels
    only: the trajectory is then the fixed unitary circuit ``branch_circuit``)."""
    for _, ch in sites(channels_after, len(circ.gates)):
        if fixed_weights(ch[0], ch[1]) is None:
            raise ValueError("gradients need Pauli or depolarizing channels")
    _, choices, margins = trajectory(circ, params, channels_after, seed, t)
    bc = branch_circuit(circ, channels_after, choices)
    e, g = O.adjoint_gradient(bc, ham, params, O.zero_state(circ.n_qubits))
    return e, g, choices, margins


def enumerate_branches(circ: Circuit, params, channels_after: Dict[int, list]):
    """Every branch sequence with its probability (brute force, few sites):
    [(probability, final normalised state)].  The probability-weighted sum of
    |psi><psi| is the density matrix of the noisy circuit."""
    n = circ.n_qubits
    items = [("site", ch) for ch in channels_after.get(-1, [])]
    for gi, g in enumerate(circ.gates):
        items.append(("gate", g))
        items += [("site", ch) for ch in channels_after.get(gi, [])]
    out = []

    def rec(k, psi, prob):
        if prob == 0.0:
            return
        if k == len(items):
            out.append((prob, psi))
            return
        kind, obj = items[k]
        if kind == "gate":
            rec(k + 1, O.apply_gate(psi, n, O.gate_unitary(obj, params), list(obj.targets), list(obj.ctrls)), prob)
            return
        w = branch_weights(obj, psi, n)
        for i, wi in enumerate(w):
            if wi > 0:
                rec(k + 1, O.apply_gate(psi, n, branch_operator(obj, psi, n, i, w), [obj[2]]), prob * wi)

    rec(0, O.zero_state(n), 1.0)
    return out
