"""Pins of the Monte-Carlo trajectory oracle (§3.3): the probability-weighted
sum over every branch sequence equals the density matrix of the density-matrix
oracle (every channel kind, custom Kraus sets included), so each branch rule is
unbiased; Pauli-channel gradients enumerated the same way equal finite
differences of the exact noisy energy; zero-probability channels leave the
noiseless state; sampled branch frequencies follow the channel probabilities;
and the sample mean of the energy converges to tr(rho H)."""
import math

import numpy as np
import pytest

from oracle import dm_oracle as D
from oracle import qsim_oracle as O
from oracle import traj_oracle as T
from paper_2406_17248_gb300 import inputs as I


def _random_kraus(seed):
    # a 3-operator Kraus set from a random 6x2 isometry (rows split in 2x2 blocks)
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(6, 2)) + 1j * rng.normal(size=(6, 2))
    q, _ = np.linalg.qr(a)
    return [q[2 * i:2 * i + 2, :] for i in range(3)]


def _dm_run(circ, params, ch, n):
    # the density-matrix oracle, with custom Kraus sets ("kraus", (), q, mats) too
    rho = D.zero_dm(n)

    def site(rho, c):
        mats = c[3] if c[0] == "kraus" else D.channel_kraus(c[0], c[1])
        return D.apply_channel(rho, n, mats, c[2])

    for c in ch.get(-1, []):
        rho = site(rho, c)
    for i, g in enumerate(circ.gates):
        rho = D.apply_unitary(rho, n, O.gate_unitary(g, params), g.targets, g.ctrls)
        for c in ch.get(i, []):
            rho = site(rho, c)
    return rho


def _noisy_case():
    n = 3
    circ = I.hea_circuit(n, 1)
    params = I.uniform_params(circ.n_params, 5)
    ch = {-1: [("amplitude_damping", (0.2,), 1)],
          1: [("depolarizing", (0.3,), 0)],
          4: [("pauli", (0.1, 0.05, 0.2), 2)],
          6: [("phase_damping", (0.35,), 1)],
          len(circ.gates) - 1: [("kraus", (), 0, _random_kraus(1))]}
    return n, circ, params, ch


def test_enumerated_branches_reproduce_the_density_matrix():
    n, circ, params, ch = _noisy_case()
    br = T.enumerate_branches(circ, params, ch)
    assert sum(p for p, _ in br) == pytest.approx(1.0, abs=1e-12)
    rho = sum(p * np.outer(s, s.conj()) for p, s in br)
    np.testing.assert_allclose(rho, _dm_run(circ, params, ch, n), atol=1e-12)
    for _, s in br:
        assert np.linalg.norm(s) == pytest.approx(1.0, abs=1e-12)


def test_enumerated_pauli_gradients_match_exact_noisy_energy():
    n = 3
    circ = I.hea_circuit(n, 1)
    ham = I.chain_zz_x(n, 0.7)
    params = I.uniform_params(circ.n_params, 8)
    ch = {0: [("depolarizing", (0.2,), 0)], 3: [("pauli", (0.1, 0.0, 0.3), 1)]}
    # exact noisy energy and its central differences
    def exact(x):
        return D.expectation(D.run(circ, x, ch, n), ham)
    h = 1e-6
    fd = np.array([(exact(params + h * e) - exact(params - h * e)) / (2 * h) for e in np.eye(circ.n_params)])
    # branch-weighted adjoint gradients of the branch circuits
    st = T.sites(ch, len(circ.gates))
    ws = [T.fixed_weights(c[0], c[1]) for _, c in st]
    g = np.zeros(circ.n_params)
    e = 0.0
    for a in range(4):
        for b in range(4):
            p = ws[0][a] * ws[1][b]
            if p == 0:
                continue
            bc = T.branch_circuit(circ, ch, [a, b])
            eb, gb = O.adjoint_gradient(bc, ham, params, O.zero_state(n))
            e += p * eb
            g += p * gb
    assert e == pytest.approx(exact(params), abs=1e-12)
    np.testing.assert_allclose(g, fd, atol=1e-7)


def test_zero_probability_channels_are_noiseless():
    n = 4
    circ = I.hea_circuit(n, 2)
    params = I.uniform_params(circ.n_params, 3)
    ch = {i: [("depolarizing", (0.0,), i % n), ("amplitude_damping", (0.0,), (i + 1) % n)] for i in range(0, 20, 4)}
    psi, choices, _ = T.trajectory(circ, params, ch, seed=7, t=11)
    np.testing.assert_allclose(psi, O.evolve(circ, params, O.zero_state(n)), atol=1e-13)
    assert choices == [0] * len(choices)


def test_branch_frequencies_follow_probabilities():
    circ = I.Circuit(1, [I.Gate("H", (0,))], 0)
    ch = {0: [("pauli", (0.3, 0.1, 0.0), 0)]}
    n_t = 4000
    counts = np.zeros(4)
    for t in range(n_t):
        _, c, _ = T.trajectory(circ, [], ch, seed=123, t=t)
        counts[c[0]] += 1
    for i, p in enumerate((0.6, 0.3, 0.1, 0.0)):
        sd = math.sqrt(p * (1 - p) / n_t)
        assert abs(counts[i] / n_t - p) <= 4 * sd + 1e-12


def test_state_dependent_branch_frequencies():
    # amplitude damping of |1>: the decay branch has probability gamma
    circ = I.Circuit(1, [I.Gate("X", (0,))], 0)
    ch = {0: [("amplitude_damping", (0.35,), 0)]}
    n_t = 3000
    decays = sum(T.trajectory(circ, [], ch, seed=5, t=t)[1][0] for t in range(n_t))
    assert abs(decays / n_t - 0.35) <= 4 * math.sqrt(0.35 * 0.65 / n_t)


def test_sample_mean_converges_to_density_matrix_energy():
    n = 4
    circ = I.hea_circuit(n, 2)
    params = I.uniform_params(circ.n_params, 9)
    ham = I.chain_zz_x(n, 0.5)
    ch = {i: [("depolarizing", (0.05,), i % n), ("amplitude_damping", (0.1,), (i + 2) % n)]
          for i in range(0, len(circ.gates), 3)}
    exact = D.expectation(D.run(circ, params, ch, n), ham)
    es = np.array([O.expectation(T.trajectory(circ, params, ch, seed=2, t=t)[0], ham) for t in range(1500)])
    assert abs(es.mean() - exact) < 5 * es.std() / math.sqrt(es.size)


def test_choose_rule():
    assert T.choose([0.5, 0.5], 0.0) == 0
    assert T.choose([0.0, 1.0], 0.0) == 1
    assert T.choose([0.25, 0.25, 0.5], 0.5) == 2
    assert T.choose([0.25, 0.25, 0.5], 0.4999) == 1
