"""Pins of the FP64 oracle to values the paper prints (tests/golden/*.json).

Each golden entry carries its citation.  A plausible mistake in the oracle
(a sign, a half-angle, an endianness or layer-order slip) breaks one of these.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import least_squares, minimize

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_qupack_qaoa_k5_expectation_and_gradients():
    """§6.2.2: K5, depth 10, gamma = 1, beta = 2 -> printed E and 20 gradients."""
    g = _load("qupack_qaoa_k5.json")
    n, p = g["n_qubits"], g["depth"]
    E, dg, db = O.qaoa_expectation_with_grad(n, I.complete_graph(n), [g["gamma"]] * p, [g["beta"]] * p, 1.0)
    assert abs(E - g["expectation"]) < 1e-12
    np.testing.assert_allclose(dg, g["gamma_grad"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(db, g["beta_grad"], rtol=0, atol=1e-10)


def test_qupack_qaoa_k5_through_gate_level_circuit():
    """The same pin through the generic gate path: RZZ(2 gamma) per edge, RX(beta)
    per qubit, adjoint gradient chained through shared parameters."""
    g = _load("qupack_qaoa_k5.json")
    n, p = g["n_qubits"], g["depth"]
    edges = I.complete_graph(n)
    circ = I.qaoa_circuit(n, edges, p, gamma_coef=2.0)
    ham = I.maxcut_zz(n, edges)
    params = np.array([g["gamma"]] * p + [g["beta"]] * p)
    E, grad = O.adjoint_gradient(circ, ham, params, O.zero_state(n))
    assert abs(E - g["expectation"]) < 1e-12
    np.testing.assert_allclose(grad[:p], g["gamma_grad"], atol=1e-10)
    np.testing.assert_allclose(grad[p:], g["beta_grad"], atol=1e-10)


def test_zz_after_rx_printed_value():
    g = _load("paper_prints.json")["zz_after_rx"]
    circ = I.Circuit(2, [I.Gate("RX", (0,), const=g["theta"])])
    psi = O.evolve(circ, [], O.zero_state(2))
    E = O.expectation(psi, I.pauli_sum_from_strings(2, [(1.0, "Z0 Z1")]))
    assert abs(E - g["value"]) < 1e-15


def test_inner_product_printed_value():
    g = _load("paper_prints.json")["inner_product"]
    psi = O.evolve(I.Circuit(2, [I.Gate("RX", (0,), const=g["rx"])]), [], O.zero_state(2))
    phi = O.evolve(I.Circuit(2, [I.Gate("RY", (0,), const=g["ry"])]), [], O.zero_state(2))
    ip = O.inner_product(phi, psi)
    assert abs(ip.real - g["re"]) < 1e-15 and abs(ip.imag - g["im"]) < 1e-15


def test_apply_hamiltonian_then_circuit_printed_state():
    """§2.6.1: little endian, X.on(target, control) order, Y = [[0,-i],[i,0]]."""
    g = _load("paper_prints.json")["apply_hamiltonian_then_circuit"]
    ham = I.pauli_sum_from_strings(2, [(1.0, "X0 Y1")])
    psi = O.apply_hamiltonian(O.zero_state(2), ham)
    circ = I.Circuit(2, [I.Gate("H", (0,)), I.Gate("X", (1,), (0,))])
    psi = O.evolve(circ, [], psi)
    np.testing.assert_allclose(psi.real, g["amplitudes_re"], atol=1e-15)
    np.testing.assert_allclose(psi.imag, g["amplitudes_im"], atol=1e-15)


def test_operator_matrix_printed():
    g = _load("paper_prints.json")["operator_matrix"]
    ham = I.pauli_sum_from_strings(2, [tuple(t) for t in g["terms"]])
    M = O.hamiltonian_matrix(ham)
    np.testing.assert_array_equal(M.real, np.array(g["re"], float))
    np.testing.assert_array_equal(M.imag, np.array(g["im"], float))


def _rotation_ansatz():
    # §4.1.1: rz('c',0).rx(pi/2,0).rz('a',0).rx(-pi/2,0).rz('b',0); parameter order (c, a, b)
    return I.Circuit(1, [I.Gate("RZ", (0,), param=0), I.Gate("RX", (0,), const=math.pi / 2),
                         I.Gate("RZ", (0,), param=1), I.Gate("RX", (0,), const=-math.pi / 2),
                         I.Gate("RZ", (0,), param=2)], 3)


def _rotation_fit_residual(grad_scale=1.0):
    g = _load("paper_prints.json")["learning_rotation"]
    circ = _rotation_ansatz()
    ham = I.pauli_sum_from_strings(1, [(1.0, "X0")])
    target = np.array([g["f"], g["grad"][1], g["grad"][2]])

    def resid(ab):
        E, gr = O.adjoint_gradient(circ, ham, [0.3, ab[0], ab[1]], O.zero_state(1))
        return np.array([E, grad_scale * gr[1], grad_scale * gr[2]]) - target

    best = None
    for a0 in np.linspace(-3, 3, 7):
        for b0 in np.linspace(-3, 3, 7):
            r = least_squares(resid, [a0, b0], xtol=1e-15, ftol=1e-15, gtol=1e-15)
            if best is None or r.cost < best.cost:
                best = r
    return best


def test_learning_rotation_gradient_consistent_with_print():
    """§4.1.1 prints f and three gradients at an unprinted random point: three
    equations in the two effective unknowns (a, b) must be consistent, and the
    gradient in c (a phase on |0>) must vanish."""
    best = _rotation_fit_residual()
    assert np.max(np.abs(best.fun)) < 2e-8
    circ = _rotation_ansatz()
    ham = I.pauli_sum_from_strings(1, [(1.0, "X0")])
    for c in (-2.0, 0.1, 1.7):
        _, gr = O.adjoint_gradient(circ, ham, [c, best.x[0], best.x[1]], O.zero_state(1))
        assert abs(gr[0]) < 1e-15


def test_learning_rotation_detects_dropped_half_angle():
    """Planted mistake (in the oracle's output, on the CPU): a gradient off by the
    half-angle factor no longer fits the printed numbers."""
    best = _rotation_fit_residual(grad_scale=2.0)
    assert np.max(np.abs(best.fun)) > 1e-4


def test_qaoa_5node_p4_optimum_cut():
    """§5.2: p = 4 QAOA on the 5-node, 6-edge graph reaches cut 4.939257.
    Multi-start BFGS on the oracle's adjoint gradient finds the same optimum."""
    g = _load("paper_prints.json")["qaoa_5node_p4"]
    edges = [tuple(e) for e in g["edges"]]
    n, p = 5, g["p"]

    def f(x):
        E, dg, db = O.qaoa_expectation_with_grad(n, edges, x[:p], x[p:], 0.5)
        return E, np.concatenate([dg, db])

    rng = np.random.default_rng(0)
    best = -1.0
    for _ in range(40):
        r = minimize(f, rng.uniform(0, np.pi, 2 * p), jac=True, method="BFGS")
        best = max(best, (len(edges) - r.fun) / 2)
    assert abs(best - g["cut"]) < g["print_precision"]
    assert O.maxcut_brute_force(n, edges) == 5


@pytest.mark.parametrize("gs", [0.5, 1.0])
def test_qaoa_p1_closed_form_matches_simulation(gs):
    """The published depth-1 MaxCut formula (any n, triangles included) against
    the simulated energy; the GPU tests use the same formula at 30 qubits."""
    graphs = [(8, I.random_regular_graph(8, 3, 1)), (9, I.erdos_renyi(9, 0.5, 2)), (7, I.complete_graph(7)),
              (10, I.erdos_renyi(10, 0.4, 5))]
    for n, e in graphs:
        for g, b in [(0.7, 0.3), (-1.1, 2.0), (2.5, -0.4)]:
            E = O.qaoa_expectation_with_grad(n, e, [g], [b], gamma_scale=gs)[0]
            assert abs(E - O.qaoa_p1_energy_closed_form(n, e, g, b, gs)) < 1e-12
