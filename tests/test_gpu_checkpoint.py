"""Adjoint state checkpoints (the forward sweep saves psi every K gates or
layers; the reverse sweep reloads it there instead of the uncomputed state):
results equal the oracle with checkpoints on, the input state is restored, the
complex64 drift of a long uncompute chain is no larger than without them, and
the QAOA engine with checkpoints reproduces the stored 24-qubit oracle values.
Tolerances as in tests/test_gpu_parity.py."""
import json
import os

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = {0: 5e-5, 1: 1e-11}
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


def scale(ham):
    return max(1.0, float(np.abs(ham.coef).sum()))


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
    tol = TOL[dt] * scale(ham)
    assert abs(E - E0) < tol and np.abs(g - G0).max() < tol
    assert np.abs(psi.get_qs() - psi0).max() < TOL[dt] * 10
    # a list of Hamiltonians reuses the checkpoints for every reverse sweep
    hams = [ham, I.chain_zz_x(n, 0.3)]
    psi.set_qs(psi0)
    Es, Gs = Q.expectation_with_grad_multi(psi, lam, c, [Q.Hamiltonian(h) for h in hams], x)
    for h, e, gg in zip(hams, Es, Gs):
        e0, g0 = O.adjoint_gradient(circ, h, x, psi0)
        assert abs(e - e0) < TOL[dt] * scale(h) and np.abs(gg - g0).max() < TOL[dt] * scale(h)


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
        assert abs(E - E0) < TOL[0] * scale(ham)
    assert errs[256] < TOL[0] * scale(ham)
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
        tol = TOL[dt] * len(edges)
        assert abs(E - g["energy"]) < tol
        assert np.abs(dg - g["dgamma"]).max() < tol
        assert np.abs(db - g["dbeta"]).max() < tol
