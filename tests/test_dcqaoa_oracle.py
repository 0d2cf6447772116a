"""Pins of the DC-QAOA oracle (§5.4): the gate-level ansatz against the
definition by matrix exponentials, the gamma = 0 closed form, the ground energy
of the Ising chain by enumeration, the adjoint gradient against central
differences, and the paper's observation that one DC-QAOA layer reaches the
exact ground energy of the 12-qubit longitudinal-field chain under Adam while
one plain QAOA layer stays far above it."""
import math

import numpy as np
import pytest

from oracle import gnn_oracle as G
from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_chain_ground_energy_closed_form_and_spectrum(n):
    rng = np.random.default_rng(n)
    J, h = float(rng.uniform(0.2, 2)), float(rng.uniform(0.2, 2))
    brute = O.ising_chain_min_energy_brute_force(n, J, h)
    assert brute == pytest.approx(-(J * (n - 1) + h * n), abs=1e-12)
    evals = np.linalg.eigvalsh(O.hamiltonian_matrix(I.lfim(n, J, h)))
    assert evals[0] == pytest.approx(brute, abs=1e-10)


@pytest.mark.parametrize("n,p,cd", [(3, 1, True), (4, 2, True), (6, 3, True), (5, 2, False)])
def test_gate_level_ansatz_equals_definition(n, p, cd):
    rng = np.random.default_rng(10 * n + p)
    J, h = float(rng.uniform(0.5, 1.5)), float(rng.uniform(0.5, 1.5))
    circ = I.dcqaoa_circuit(n, p, J, h, cd=cd)
    x = rng.uniform(-np.pi, np.pi, circ.n_params)
    got = O.evolve(circ, x, O.zero_state(n))
    want = O.dcqaoa_state_by_definition(n, I.lfim(n, J, h), x, p, cd=cd)
    np.testing.assert_allclose(got, want, atol=1e-12)
    # the dense Kronecker-product applier agrees too
    np.testing.assert_allclose(O.dense_circuit_unitary(circ, x) @ O.zero_state(n), want, atol=1e-12)


def test_transverse_term_is_a_first_order_product():
    # k != 0: the X term does not commute with the Z terms, so the gate-level
    # U_p is the product of the three term exponentials (the toolkit's
    # first-order decomposition), not exp(-i gamma H_prob); it matches the
    # definition only as gamma -> 0, with an O(gamma^2) error.
    n = 4
    circ = I.dcqaoa_circuit(n, 1, 1.0, 1.0, k=0.7)
    errs = []
    for g in (0.1, 0.05):
        x = np.array([g, 0.3, -0.2])
        d = O.evolve(circ, x, O.zero_state(n)) - O.dcqaoa_state_by_definition(n, I.lfim(n, 1.0, 1.0, 0.7), x, 1)
        errs.append(np.linalg.norm(d))
    assert errs[0] > 1e-4
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)


@pytest.mark.parametrize("n", [6, 12])
def test_gamma0_closed_form(n):
    ham = I.lfim(n)
    circ = I.dcqaoa_circuit(n, 1)
    for beta, alpha in ((0.0, 0.0), (0.37, -0.2), (-1.1, 0.9), (0.5, -math.pi / 4)):
        e = O.expectation_of_circuit(circ, ham, [0.0, beta, alpha], O.zero_state(n))
        assert e == pytest.approx(O.dcqaoa_p1_energy_at_gamma0(n, 1.0, 1.0, alpha), abs=1e-12)
    e = O.expectation_of_circuit(circ, ham, [0.0, 0.3, -math.pi / 4], O.zero_state(n))
    assert e == pytest.approx(-(2 * n - 1), abs=1e-12)


def test_no_evolution_without_mixing():
    # beta = alpha = 0: U_p is diagonal, so every Z expectation keeps its |+> value 0.
    n = 7
    x = [0.83, 0.0, 0.0]
    assert O.expectation_of_circuit(I.dcqaoa_circuit(n, 1), I.lfim(n), x, O.zero_state(n)) == pytest.approx(0, abs=1e-12)


def test_adjoint_gradient_matches_central_differences():
    n, p = 6, 2
    circ = I.dcqaoa_circuit(n, p, 1.0, 0.8)
    ham = I.lfim(n, 1.0, 0.8)
    x = np.random.default_rng(3).uniform(-1, 1, circ.n_params)
    e, g = O.adjoint_gradient(circ, ham, x, O.zero_state(n))
    fd = O.finite_difference_gradient(circ, ham, x, O.zero_state(n))
    np.testing.assert_allclose(g, fd, atol=1e-7)
    assert e == pytest.approx(O.expectation_of_circuit(circ, ham, x, O.zero_state(n)), abs=1e-12)


def _adam_energies(cd, steps, seed):
    n = 12
    circ = I.dcqaoa_circuit(n, 1, cd=cd)
    ham = I.lfim(n)
    x = np.random.default_rng(seed).uniform(0.0, 0.1, circ.n_params)
    m, v = np.zeros_like(x), np.zeros_like(x)
    hist = []
    for t in range(1, steps + 1):
        e, g = O.adjoint_gradient(circ, ham, x, O.zero_state(n))
        hist.append(e)
        x, m, v = G.adam(x, m, v, g, t, 0.05)
    return np.array(hist)


def test_paper_observation_dcqaoa_reaches_ground_qaoa_trapped():
    # 12-qubit LFIM (J = h = 1, k = 0), one layer, Adam with learning rate 0.05:
    # DC-QAOA converges to the exact ground energy -23 while QAOA stays trapped.
    dc = _adam_energies(True, 100, 1)
    qa = _adam_energies(False, 100, 1)
    assert dc[-1] == pytest.approx(-23.0, abs=1e-3)
    assert qa.min() > -12.0
