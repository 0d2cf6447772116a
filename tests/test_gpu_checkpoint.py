"""Adjoint state checkpoints (the forward sweep saves psi every K gates or
layers; the reverse sweep reloads it there instead of the uncomputed state):
results equal the oracle with checkpoints on, the input state is restored, the
complex64 drift of a long uncompute chain is no larger than without them, and
the QAOA engine with checkpoints reproduces the stored 24-qubit oracle values.
Tolerances: the rule of tests/tolerance.py."""
import json
import os

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

from tolerance import TOL, check, energy_tol, grad_tol, qaoa_grad_tols, state_err

pytestmark = pytest.mark.gpu
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


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("k", [1, 7, 40])
def test_gradients_with_checkpoints(Q, dt, k):
    n = 14
    circ = I.random_mixed_circuit(n, 120, 5, max_ctrls=2, with_matrix=True)
    ham = I.random_pauli_sum(n, 8, 3)
    x = I.uniform_params(circ.n_params, 4)
    psi0 = I.random_state(n, 6)
    E0, G0 = O.adjoint_gradient(circ, ham, x, psi0)
    c = Q.circuit_from(circ).finalize(dt, tile_bits=8, checkpoint=k)
    psi, lam = Q.State(n, dt), Q.State(n, dt)
    psi.set_qs(psi0)
    E, g = Q.expectation_with_grad(psi, lam, c, Q.Hamiltonian(ham), x)
    tag = f"checkpoint k={k} dt={dt}"
    check(tag + " energy", abs(E - E0), energy_tol(dt, ham))
    check(tag + " grad", np.abs(g - G0), grad_tol(dt, ham, circ))
    check(tag + " restored psi", state_err(psi.get_qs(), psi0), 2 * TOL[dt])
    # a list of Hamiltonians reuses the checkpoints for every reverse sweep
    hams = [ham, I.chain_zz_x(n, 0.3)]
    psi.set_qs(psi0)
    Es, Gs = Q.expectation_with_grad_multi(psi, lam, c, [Q.Hamiltonian(h) for h in hams], x)
    for h, e, gg in zip(hams, Es, Gs):
        e0, g0 = O.adjoint_gradient(circ, h, x, psi0)
        check(tag + " multi energy", abs(e - e0), energy_tol(dt, h))
        check(tag + " multi grad", np.abs(gg - g0), grad_tol(dt, h, circ))


def test_checkpoints_bound_complex64_drift(Q):
    # 16 qubits, 2816 gates (HEA depth 64): the uncomputed psi of the reverse
    # sweep drifts from the forward states in complex64; reloading it every 256
    # gates keeps the gradient at least as close to the FP64 oracle
    n = 16
    circ = I.hea_circuit(n, 64)
    ham = I.chain_zz_x(n, 0.5)
    x = I.uniform_params(circ.n_params, 9)
    E0, G0 = O.adjoint_gradient(circ, ham, x, O.zero_state(n))
    errs = {}
    for k in (0, 256):
        c = Q.circuit_from(circ).finalize(0, checkpoint=k)
        psi, lam = Q.State(n, 0), Q.State(n, 0)
        psi.set_basis(0)
        E, g = Q.expectation_with_grad(psi, lam, c, Q.Hamiltonian(ham), x)
        errs[k] = float(np.abs(g - G0).max())
        check(f"hea16 depth64 energy checkpoint={k}", abs(E - E0), energy_tol(0, ham))
        check(f"hea16 depth64 grad checkpoint={k}", np.abs(g - G0), grad_tol(0, ham, circ))
    assert errs[256] <= errs[0] * 1.05 + 1e-7, errs


@pytest.mark.parametrize("k", [1, 3])
def test_qaoa_checkpoints_against_stored_oracle_values(Q, k):
    g = json.load(open(os.path.join(GOLD, "qaoa24_p8.json")))
    n, p = g["n"], g["p"]
    edges = [tuple(e) for e in g["edges"]]
    for dt in (0, 1):
        q = Q.QAOA(n, edges, p, gamma_scale=g["gamma_scale"], dtype=dt, checkpoint=k)
        psi, lam = Q.State(n, dt), Q.State(n, dt)
        E, dg, db = q.expectation_with_grad(psi, lam, g["gamma"], g["beta"])
        te, tg, tb = qaoa_grad_tols(dt, n, len(edges), g["gamma_scale"])
        check(f"qaoa24 checkpoint={k} energy dt={dt}", abs(E - g["energy"]), te)
        check(f"qaoa24 checkpoint={k} dgamma dt={dt}", np.abs(np.array(dg) - g["dgamma"]), tg)
        check(f"qaoa24 checkpoint={k} dbeta dt={dt}", np.abs(np.array(db) - g["dbeta"]), tb)
