"""Pins of the FP64 oracle to closed forms, brute force and independent algorithms."""
import math

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

ALL_1Q = ["I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "PS"]
ALL_2Q = ["SWAP", "RXX", "RYY", "RZZ"]


@pytest.mark.parametrize("kind", ALL_1Q + ALL_2Q)
def test_unitarity(kind):
    U = O.gate_matrix(kind, 0.7311)
    np.testing.assert_allclose(U @ U.conj().T, np.eye(U.shape[0]), atol=1e-15)


@pytest.mark.parametrize("kind", ["RX", "RY", "RZ", "PS", "RXX", "RYY", "RZZ"])
def test_derivative_matrix_matches_finite_difference(kind):
    t, h = 0.918, 1e-6
    fd = (O.gate_matrix(kind, t + h) - O.gate_matrix(kind, t - h)) / (2 * h)
    np.testing.assert_allclose(O.gate_matrix_derivative(kind, t), fd, atol=1e-9)


def test_gate_identities():
    H, X, Z = (O.gate_matrix(k) for k in "HXZ")
    np.testing.assert_allclose(H @ X @ H, Z, atol=1e-15)
    # CNOT^2 = I and RZZ(t) = CNOT . RZ(t)_target . CNOT, via the dense applier
    t = 1.234
    cnot = O.dense_gate_unitary(2, X, (1,), (0,))
    np.testing.assert_allclose(cnot @ cnot, np.eye(4), atol=1e-15)
    rz = O.dense_gate_unitary(2, O.gate_matrix("RZ", t), (1,))
    rzz = O.dense_gate_unitary(2, O.gate_matrix("RZZ", t), (0, 1))
    np.testing.assert_allclose(cnot @ rz @ cnot, rzz, atol=1e-15)
    # S = T^2, Z = S^2, RZ(t) = e^{-it/2} PS(t)
    np.testing.assert_allclose(O.gate_matrix("T") @ O.gate_matrix("T"), O.gate_matrix("S"), atol=1e-15)
    np.testing.assert_allclose(O.gate_matrix("S") @ O.gate_matrix("S"), Z, atol=1e-15)
    np.testing.assert_allclose(O.gate_matrix("RZ", t), np.exp(-0.5j * t) * O.gate_matrix("PS", t), atol=1e-15)


def test_rotations_are_exponentials_of_paulis():
    from scipy.linalg import expm
    t = -2.1
    for k, P in (("RX", O._X), ("RY", O._Y), ("RZ", O._Z)):
        np.testing.assert_allclose(O.gate_matrix(k, t), expm(-0.5j * t * P), atol=1e-14)
    for k, P in (("RXX", O._X), ("RYY", O._Y), ("RZZ", O._Z)):
        np.testing.assert_allclose(O.gate_matrix(k, t), expm(-0.5j * t * np.kron(P, P)), atol=1e-14)


def test_bell_and_ghz_closed_forms():
    for n in (2, 3, 5, 8):
        gates = [I.Gate("H", (0,))] + [I.Gate("X", (q,), (q - 1,)) for q in range(1, n)]
        psi = O.evolve(I.Circuit(n, gates), [], O.zero_state(n))
        want = np.zeros(1 << n, complex)
        want[0] = want[-1] = 1 / math.sqrt(2)
        np.testing.assert_allclose(psi, want, atol=1e-15)


@pytest.mark.parametrize("theta", [-2.9, -0.3, 0.0, 1.1, 3.0])
def test_ry_expectations_closed_form(theta):
    psi = O.evolve(I.Circuit(1, [I.Gate("RY", (0,), const=theta)]), [], O.zero_state(1))
    z = O.expectation(psi, I.pauli_sum_from_strings(1, [(1.0, "Z0")]))
    x = O.expectation(psi, I.pauli_sum_from_strings(1, [(1.0, "X0")]))
    assert abs(z - math.cos(theta)) < 1e-15 and abs(x - math.sin(theta)) < 1e-15


def _random_mixed_circuit(n, n_gates, seed):
    return I.random_mixed_circuit(n, n_gates, seed)


@pytest.mark.parametrize("seed", range(6))
def test_axis_applier_matches_dense_applier(seed):
    n = 2 + seed  # 2..7
    circ = _random_mixed_circuit(n, 25, seed)
    params = np.random.default_rng(100 + seed).uniform(-3, 3, circ.n_params)
    psi0 = np.random.default_rng(seed).normal(size=1 << n) + 0j
    psi0 /= np.linalg.norm(psi0)
    W = O.dense_circuit_unitary(circ, params)
    np.testing.assert_allclose(O.evolve(circ, params, psi0), W @ psi0, atol=1e-13)
    np.testing.assert_allclose(W @ W.conj().T, np.eye(1 << n), atol=1e-13)


def test_norm_preserved_and_inverse_restores():
    n = 9
    circ = I.random_circuit(n, 200, seed=7)
    psi = O.evolve(circ, [], O.zero_state(n))
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    inv = [I.Gate("MATRIX", g.targets, g.ctrls,
                  matrix=tuple(O.gate_unitary(g, []).conj().T.reshape(-1))) for g in reversed(circ.gates)]
    back = O.evolve(I.Circuit(n, inv), [], psi)
    np.testing.assert_allclose(back, O.zero_state(n), atol=1e-13)


def _random_pauli_sum(n, n_terms, seed):
    return I.random_pauli_sum(n, n_terms, seed)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_pauli_action_and_expectation_match_dense(n):
    ham = _random_pauli_sum(n, 12, n)
    rng = np.random.default_rng(n)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    Hm = O.hamiltonian_matrix(ham)
    np.testing.assert_allclose(O.apply_hamiltonian(psi, ham), Hm @ psi, atol=1e-12)
    assert abs(O.expectation(psi, ham) - np.real(np.vdot(psi, Hm @ psi))) < 1e-12
    np.testing.assert_allclose(Hm, Hm.conj().T, atol=1e-15)


def test_adjoint_matches_parameter_shift_hea():
    n = 5
    circ = I.hea_circuit(n, 3)
    ham = I.chain_zz_x(n)
    params = I.uniform_params(circ.n_params, seed=1)
    E, g_adj = O.adjoint_gradient(circ, ham, params, O.zero_state(n))
    g_ps = O.parameter_shift_gradient(circ, ham, params, O.zero_state(n))
    np.testing.assert_allclose(g_adj, g_ps, atol=1e-12)
    assert abs(E - O.expectation_of_circuit(circ, ham, params, O.zero_state(n))) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_adjoint_matches_finite_difference_controlled_and_shared(seed):
    n = 4
    circ = _random_mixed_circuit(n, 30, 50 + seed)
    # share parameters: fold every parameter index onto 3 shared ones
    gates = [I.Gate(g.kind, g.targets, g.ctrls, (g.param % 3) if g.param >= 0 else -1, g.coef, g.const, g.matrix)
             for g in circ.gates]
    circ = I.Circuit(n, gates, 3)
    ham = _random_pauli_sum(n, 6, seed)
    params = np.random.default_rng(seed).uniform(-3, 3, 3)
    psi0 = O.plus_state(n)
    _, g_adj = O.adjoint_gradient(circ, ham, params, psi0)
    g_fd = O.finite_difference_gradient(circ, ham, params, psi0, h=1e-5)
    np.testing.assert_allclose(g_adj, g_fd, atol=1e-7)


def test_qaoa_layer_form_matches_gate_form():
    n, p = 6, 3
    edges = I.random_regular_graph(n, 3, seed=3)
    rng = np.random.default_rng(3)
    gam, bet = rng.uniform(0, np.pi, p), rng.uniform(0, np.pi, p)
    for scale, coef in ((0.5, 1.0), (1.0, 2.0)):
        E, dg, db = O.qaoa_expectation_with_grad(n, edges, gam, bet, scale)
        circ = I.qaoa_circuit(n, edges, p, gamma_coef=coef)
        E2, g2 = O.adjoint_gradient(circ, I.maxcut_zz(n, edges), np.concatenate([gam, bet]), O.zero_state(n))
        assert abs(E - E2) < 1e-13
        np.testing.assert_allclose(np.concatenate([dg, db]), g2, atol=1e-12)
        g3 = O.parameter_shift_gradient(circ, I.maxcut_zz(n, edges), np.concatenate([gam, bet]), O.zero_state(n))
        np.testing.assert_allclose(g2, g3, atol=1e-12)


def test_cut_values_brute_force():
    n = 7
    edges = I.erdos_renyi(n, 0.5, seed=2)
    C = O.cut_values(n, edges)
    for x in range(1 << n):
        bits = [(x >> q) & 1 for q in range(n)]
        cut = sum(bits[a] != bits[b] for a, b in edges)
        assert C[x] == len(edges) - 2 * cut


def test_random_regular_graph_is_regular():
    for seed in range(3):
        edges = I.random_regular_graph(30, 3, seed)
        assert len(edges) == 45
        deg = np.bincount(np.array(edges).reshape(-1), minlength=30)
        assert np.all(deg == 3)


def test_splitmix64_published_vector():
    """splitmix64 from state 1234567: the first five outputs of the published generator."""
    s, out = 1234567, []
    for _ in range(5):
        s, z = O.splitmix64(s)
        out.append(z)
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_sampling_inverse_cdf_brute_force_and_chi_square():
    from scipy.stats import chisquare
    n = 4
    circ = I.random_circuit(n, 30, seed=11)
    psi = O.evolve(circ, [], O.zero_state(n))
    p = np.abs(psi) ** 2
    # brute force on the definition for a few shots
    got = O.sample(psi, 50, seed=99)
    for s in range(50):
        u = O.shot_uniform(99, s)
        acc, x = 0.0, 0
        while acc + p[x] <= u * p.sum() and x < len(p) - 1:
            acc += p[x]
            x += 1
        assert got[s] == x
    shots = 100000
    counts = np.bincount(O.sample(psi, shots, seed=5).astype(np.int64), minlength=1 << n)
    keep = p > 1e-12
    assert np.all(counts[~keep] == 0)
    stat = chisquare(counts[keep], p[keep] / p[keep].sum() * shots)
    assert stat.pvalue > 1e-4


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_dense_block_appliers_agree_and_factorise(k):
    """k-target unitaries (dense fused blocks): the axis applier against explicit
    Kronecker products, and a product of single-qubit unitaries U_{k-1} (x) ... (x)
    U_0 (basis index sum_b bit(targets[b]) 2^b) against applying each factor on its
    own target."""
    rng = np.random.default_rng(k)
    n = 8
    targets = list(rng.permutation(n)[:k])
    z = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    U, _ = np.linalg.qr(z)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    if k <= 4:  # explicit Kronecker sums grow as 4^k; the factorised check below covers k = 5, 6
        a = O.apply_gate(psi, n, U, targets)
        b = O.dense_gate_unitary(n, U, targets) @ psi
        assert np.max(np.abs(a - b)) < 1e-12
    singles = [np.linalg.qr(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)))[0] for _ in range(k)]
    K = np.eye(1, dtype=complex)
    for s in reversed(singles):
        K = np.kron(K, s)
    want = psi.copy()
    for t, s in zip(targets, singles):
        want = O.apply_gate(want, n, s, [t])
    assert np.max(np.abs(O.apply_gate(psi, n, K, targets) - want)) < 1e-12


def test_measure_bell_state_and_statistics():
    """A Bell pair collapses onto |00> or |11> whichever qubit is measured; over
    many seeds the outcome frequency follows P(1) (binomial, 5 sigma)."""
    bell = np.zeros(4, dtype=complex)
    bell[0] = bell[3] = 1 / math.sqrt(2)
    for q in (0, 1):
        for seed in range(8):
            o, st, p1 = O.measure(bell, 2, q, seed)
            want = np.zeros(4, dtype=complex)
            want[3 if o else 0] = 1.0
            assert abs(p1 - 0.5) < 1e-15 and np.allclose(st, want, atol=1e-15)
    psi = I.random_state(5, 3)
    _, _, p1 = O.measure(psi, 5, 2, 0)
    trials = 4000
    ones = sum(O.measure(psi, 5, 2, s)[0] for s in range(trials))
    assert abs(ones - trials * p1) < 5 * math.sqrt(trials * p1 * (1 - p1))
    o, st, _ = O.measure(psi, 5, 2, 11)
    assert abs(np.linalg.norm(st) - 1.0) < 1e-13
    assert np.all(st[((np.arange(32) >> 2) & 1) != o] == 0)
