"""GPU parity of the generalised expectation E = <phi|U_l^dag H U_r|psi> and
its complex gradient (§2.6.2, §4.1) against the oracle's product rule: the
paper's printed inner product, random circuit pairs sharing parameters (one
tile and several tiles, both precisions), the Hermitian special case against
the adjoint gradient, a parameter-free left circuit, and the input states
restored on return.  Tolerance: tol * max(1, sum |c_k|), tol 5e-5 (complex64)
and 1e-11 (complex128)."""
import json
import os

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

pytestmark = pytest.mark.gpu
from tolerance import TOL, check, energy_tol, grad_tol, state_err
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def _pair(n, seed, n_r=30, n_l=24):
    r = I.random_mixed_circuit(n, n_r, seed, max_ctrls=1, with_matrix=False)
    l = I.random_mixed_circuit(n, n_l, seed + 50, max_ctrls=1, with_matrix=False)
    k = max(r.n_params, 1)
    lg = [I.Gate(g.kind, g.targets, g.ctrls, g.param % k if g.param >= 0 else -1, g.coef, g.const) for g in l.gates]
    return r, I.Circuit(n, lg, r.n_params), I.uniform_params(r.n_params, seed + 7)


def _states(Q, n, dt, psi0, phi0):
    psi, phi, lam = Q.State(n, dt), Q.State(n, dt), Q.State(n, dt)
    psi.set_qs(psi0)
    phi.set_qs(phi0)
    return psi, phi, lam


def test_printed_inner_product(Q):
    g = json.load(open(os.path.join(GOLD, "paper_prints.json")))["inner_product"]
    ur = Q.circuit_from(I.Circuit(2, [I.Gate("RX", (0,), const=g["rx"])])).finalize(1)
    ul = Q.circuit_from(I.Circuit(2, [I.Gate("RY", (0,), const=g["ry"])])).finalize(1)
    psi, phi, lam = _states(Q, 2, 1, O.zero_state(2), O.zero_state(2))
    E, grad = Q.expectation_general(psi, phi, lam, ur, ul, Q.Hamiltonian(I.pauli_sum_from_strings(2, [(1.0, "")])), [])
    assert abs(E.real - g["re"]) < 1e-12 and abs(E.imag - g["im"]) < 1e-12


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [5, 14])
def test_random_pairs(Q, dt, n):
    r, l, x = _pair(n, 3 + n)
    ham = I.random_pauli_sum(n, 6, n)
    psi0, phi0 = I.random_state(n, 11), I.random_state(n, 12)
    E0, g0 = O.general_expectation_grad(r, l, ham, x, psi0, phi0)
    psi, phi, lam = _states(Q, n, dt, psi0, phi0)
    cr = Q.circuit_from(r).finalize(dt, tile_bits=6 if n > 6 else 0)
    cl = Q.circuit_from(l).finalize(dt, tile_bits=6 if n > 6 else 0)
    E, g = Q.expectation_general(psi, phi, lam, cr, cl, Q.Hamiltonian(ham), x)
    # a parameter read by both circuits: its bound sums the gates of both
    both = I.Circuit(n, list(r.gates) + list(l.gates), max(r.n_params, l.n_params))
    tag = f"general n={n} dt={dt}"
    check(tag + " energy", abs(E - E0), energy_tol(dt, ham))
    check(tag + " grad", np.abs(g - g0), grad_tol(dt, ham, both))
    # inputs restored (forward and reverse sweeps: 2 tol)
    check(tag + " restored psi", state_err(psi.get_qs(), psi0), 2 * TOL[dt])
    check(tag + " restored phi", state_err(phi.get_qs(), phi0), 2 * TOL[dt])


@pytest.mark.parametrize("dt", [0, 1])
def test_hermitian_case_and_default_left(Q, dt):
    n = 9
    circ = I.hea_circuit(n, 2)
    ham = I.chain_zz_x(n, 0.5)
    x = I.uniform_params(circ.n_params, 2)
    c = Q.circuit_from(circ).finalize(dt)
    psi, phi, lam = _states(Q, n, dt, O.zero_state(n), O.zero_state(n))
    E, g = Q.expectation_general(psi, phi, lam, c, None, Q.Hamiltonian(ham), x)
    E0, g0 = O.adjoint_gradient(circ, ham, x, O.zero_state(n))
    tag = f"general hermitian dt={dt}"
    check(tag + " energy", abs(E - E0), energy_tol(dt, ham))
    check(tag + " grad", np.abs(g - g0), grad_tol(dt, ham, circ))
    check(tag + " energy imag", abs(E.imag), energy_tol(dt, ham))
    check(tag + " grad imag", np.abs(g.imag), grad_tol(dt, ham, circ))


def test_parameter_free_left_circuit(Q):
    n = 6
    r = I.hea_circuit(n, 1)
    l = I.random_circuit(n, 20, 4)  # fixed gates only
    ham = I.random_pauli_sum(n, 4, 1)
    x = I.uniform_params(r.n_params, 3)
    psi0, phi0 = I.random_state(n, 1), I.random_state(n, 2)
    E0, g0 = O.general_expectation_grad(r, I.Circuit(n, l.gates, r.n_params), ham, x, psi0, phi0)
    psi, phi, lam = _states(Q, n, 1, psi0, phi0)
    E, g = Q.expectation_general(psi, phi, lam, Q.circuit_from(r).finalize(1), Q.circuit_from(l).finalize(1),
                                 Q.Hamiltonian(ham), x)
    check("general fixed left energy", abs(E - E0), energy_tol(1, ham))
    check("general fixed left grad", np.abs(g - g0), grad_tol(1, ham, r))
    check("general fixed left restored phi", state_err(phi.get_qs(), phi0), 2 * TOL[1])
