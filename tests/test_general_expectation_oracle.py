"""Pins of the generalised expectation E = <phi|U_l^dag H U_r|psi> (§2.6.2,
§4.1): the paper's printed inner product (H = I, U_r = RX(2.5), U_l = RY(1.5)),
the Hermitian special case (U_l = U_r, phi = psi) against the adjoint method,
the projector observable H = |0><0| giving |<0|U_r|psi>|^2 as the paper states,
and the product-rule gradient against central differences of the complex E
(parameters shared between the two circuits included)."""
import json
import os

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _mixed_pair(n, seed):
    rng = np.random.default_rng(seed)
    r = I.random_mixed_circuit(n, 18, seed, max_ctrls=1, with_matrix=False)
    l = I.random_mixed_circuit(n, 14, seed + 50, max_ctrls=1, with_matrix=False)
    # share parameters: the left circuit's angles reuse the right circuit's indices
    k = max(r.n_params, 1)
    lg = [I.Gate(g.kind, g.targets, g.ctrls, g.param % k if g.param >= 0 else -1, g.coef, g.const) for g in l.gates]
    l = I.Circuit(n, lg, r.n_params)
    return r, l, rng.uniform(-np.pi, np.pi, r.n_params)


def test_printed_inner_product():
    g = json.load(open(os.path.join(GOLD, "paper_prints.json")))["inner_product"]
    ur = I.Circuit(2, [I.Gate("RX", (0,), const=g["rx"])])
    ul = I.Circuit(2, [I.Gate("RY", (0,), const=g["ry"])])
    ident = I.pauli_sum_from_strings(2, [(1.0, "")])
    E = O.general_expectation(ur, ul, ident, [], O.zero_state(2), O.zero_state(2))
    assert abs(E.real - g["re"]) < 1e-15 and abs(E.imag - g["im"]) < 1e-15


def test_hermitian_case_is_the_adjoint_gradient():
    n = 4
    circ = I.random_mixed_circuit(n, 25, 5, with_matrix=False)
    ham = I.random_pauli_sum(n, 6, 2)
    x = I.uniform_params(circ.n_params, 3)
    psi0 = I.random_state(n, 4)
    E, g = O.general_expectation_grad(circ, circ, ham, x, psi0, psi0)
    E0, g0 = O.adjoint_gradient(circ, ham, x, psi0)
    assert abs(E - E0) < 1e-12
    np.testing.assert_allclose(g, g0, atol=1e-12)


def test_projector_observable():
    n = 2
    circ = I.Circuit(n, [I.Gate("RX", (0,), param=0), I.Gate("RY", (1,), param=1), I.Gate("X", (1,), (0,))], 2)
    proj = I.pauli_sum_from_strings(n, [(0.25, ""), (0.25, "Z0"), (0.25, "Z1"), (0.25, "Z0 Z1")])  # |00><00|
    x = [0.7, -1.3]
    psi0 = I.random_state(n, 9)
    E = O.general_expectation(circ, circ, proj, x, psi0, psi0)
    assert abs(E - abs(O.evolve(circ, x, psi0)[0]) ** 2) < 1e-14


@pytest.mark.parametrize("n,seed", [(3, 1), (5, 2)])
def test_gradient_matches_central_differences(n, seed):
    r, l, x = _mixed_pair(n, seed)
    ham = I.random_pauli_sum(n, 5, seed)
    psi0, phi0 = I.random_state(n, seed + 10), I.random_state(n, seed + 20)
    E, g = O.general_expectation_grad(r, l, ham, x, psi0, phi0)
    assert abs(E - O.general_expectation(r, l, ham, x, psi0, phi0)) < 1e-13
    h = 1e-6
    fd = np.array([(O.general_expectation(r, l, ham, x + h * e, psi0, phi0)
                    - O.general_expectation(r, l, ham, x - h * e, psi0, phi0)) / (2 * h)
                   for e in np.eye(x.size)])
    np.testing.assert_allclose(g, fd, atol=1e-8)
    assert np.abs(g.imag).max() > 1e-3  # genuinely complex
