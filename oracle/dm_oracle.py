"""FP64 CPU oracle of the density-matrix simulator (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm may import this module; the product never calls it and shares no
code with it.

Written from §3.2 (density matrix: rho' = U rho U^dag, <H> = tr(rho H)) and §3.3
(quantum channels as Kraus maps Psi(rho) = sum_i K_i rho K_i^dag with
sum_i K_i^dag K_i = I; the Pauli, depolarizing, amplitude-damping and
phase-damping channels and custom Kraus channels).  rho is an explicit
2^n x 2^n complex128 matrix; gates and Kraus operators are embedded with the
state-vector oracle's explicit Kronecker products (qubit 0 right-most).

Parity: pinned in tests/test_dm_oracle.py -- pure states against the
state-vector oracle, trace preservation, closed forms of the damping channels,
the fully depolarized state, Kraus completeness.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from oracle import qsim_oracle as O
from paper_2406_17248_gb300.inputs import Circuit, PauliSum

_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)
_I = np.eye(2, dtype=complex)


def channel_kraus(kind: str, p: Sequence[float]) -> List[np.ndarray]:
    """Kraus operators of the §3.3 channels.  kind: 'pauli' (px, py, pz),
    'depolarizing' (p): (1 - p) rho + p/4 (I rho I + X rho X + Y rho Y + Z rho Z),
    'amplitude_damping' (gamma), 'phase_damping' (gamma)."""
    if kind == "pauli":
        px, py, pz = p
        return [math.sqrt(1 - px - py - pz) * _I, math.sqrt(px) * _X, math.sqrt(py) * _Y, math.sqrt(pz) * _Z]
    if kind == "depolarizing":
        (q,) = p
        return [math.sqrt(1 - q + q / 4) * _I, math.sqrt(q / 4) * _X, math.sqrt(q / 4) * _Y, math.sqrt(q / 4) * _Z]
    if kind == "amplitude_damping":
        (g,) = p
        return [np.array([[1, 0], [0, math.sqrt(1 - g)]], dtype=complex),
                np.array([[0, math.sqrt(g)], [0, 0]], dtype=complex)]
    if kind == "phase_damping":
        (g,) = p
        return [np.array([[1, 0], [0, math.sqrt(1 - g)]], dtype=complex),
                np.array([[0, 0], [0, math.sqrt(g)]], dtype=complex)]
    raise ValueError(kind)


def zero_dm(n: int) -> np.ndarray:
    rho = np.zeros((1 << n, 1 << n), dtype=complex)
    rho[0, 0] = 1.0
    return rho


def apply_unitary(rho: np.ndarray, n: int, U: np.ndarray, targets, ctrls=()) -> np.ndarray:
    W = O.dense_gate_unitary(n, U, list(targets), list(ctrls))
    return W @ rho @ W.conj().T


def apply_channel(rho: np.ndarray, n: int, kraus: Sequence[np.ndarray], qubit: int) -> np.ndarray:
    out = np.zeros_like(rho)
    for K in kraus:
        W = O._embed(n, K, [qubit])
        out += W @ rho @ W.conj().T
    return out


def expectation(rho: np.ndarray, ham: PauliSum) -> float:
    return float(np.real(np.trace(rho @ O.hamiltonian_matrix(ham))))


def run(circ: Circuit, params, channels_after: dict, n: int) -> np.ndarray:
    """rho after the circuit from |0..0><0..0|; channels_after[i] = [(kind, p, qubit)]
    applied after gate i (key -1: before the first gate)."""
    rho = zero_dm(n)
    for kind, p, q in channels_after.get(-1, []):
        rho = apply_channel(rho, n, channel_kraus(kind, p), q)
    for i, g in enumerate(circ.gates):
        rho = apply_unitary(rho, n, O.gate_unitary(g, params), g.targets, g.ctrls)
        for kind, p, q in channels_after.get(i, []):
            rho = apply_channel(rho, n, channel_kraus(kind, p), q)
    return rho
