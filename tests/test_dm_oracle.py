"""Pins of the density-matrix oracle: a noiseless circuit gives |psi><psi| of
the state-vector oracle; channels keep the trace and Hermiticity; closed forms of
amplitude and phase damping; full depolarizing leaves a maximally mixed qubit;
Kraus completeness of every channel."""
import math

import numpy as np
import pytest

from oracle import dm_oracle as D
from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

KINDS = [("pauli", (0.1, 0.05, 0.2)), ("depolarizing", (0.3,)), ("amplitude_damping", (0.4,)),
         ("phase_damping", (0.25,))]


@pytest.mark.parametrize("kind,p", KINDS)
def test_kraus_completeness(kind, p):
    K = D.channel_kraus(kind, p)
    assert np.allclose(sum(k.conj().T @ k for k in K), np.eye(2), atol=1e-15)


def test_noiseless_matches_state_vector():
    n = 4
    circ = I.random_mixed_circuit(n, 25, 3, with_matrix=True)
    params = I.uniform_params(circ.n_params, 2)
    rho = D.run(circ, params, {}, n)
    psi = O.evolve(circ, params, O.zero_state(n))
    assert np.allclose(rho, np.outer(psi, psi.conj()), atol=1e-13)
    ham = I.random_pauli_sum(n, 8, 1)
    assert abs(D.expectation(rho, ham) - O.expectation(psi, ham)) < 1e-13


def test_channels_keep_trace_and_hermiticity():
    n = 3
    circ = I.hea_circuit(n, 2)
    params = I.uniform_params(circ.n_params, 4)
    ch = {i: [(KINDS[i % 4][0], KINDS[i % 4][1], i % n)] for i in range(0, len(circ.gates), 3)}
    rho = D.run(circ, params, ch, n)
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.allclose(rho, rho.conj().T, atol=1e-14)
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12


def test_damping_closed_forms():
    # amplitude damping on |1>: population of |1> becomes 1 - gamma
    rho = np.diag([0.0, 1.0]).astype(complex)
    out = D.apply_channel(rho, 1, D.channel_kraus("amplitude_damping", (0.3,)), 0)
    assert np.allclose(out, np.diag([0.3, 0.7]), atol=1e-15)
    # phase damping on |+><+|: coherences scale by sqrt(1 - gamma), populations stay
    plus = np.full((2, 2), 0.5, dtype=complex)
    out = D.apply_channel(plus, 1, D.channel_kraus("phase_damping", (0.36,)), 0)
    assert np.allclose(out, [[0.5, 0.4], [0.4, 0.5]], atol=1e-15)
    # full depolarizing (p = 1) turns any qubit state into I/2
    psi = I.random_state(1, 2)
    out = D.apply_channel(np.outer(psi, psi.conj()), 1, D.channel_kraus("depolarizing", (1.0,)), 0)
    assert np.allclose(out, np.eye(2) / 2, atol=1e-15)
