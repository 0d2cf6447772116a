"""GPU parity of the complex64 micro-op tile passes (k_tile2.cu) against the
FP64 oracle and the interpreter kernel (fuse = 3 forces the micro-op form at these sizes): every gate kind with 0-2 controls on
register, tile and outside bits, dense two-qubit matrices, the adjoint reverse
passes with shared parameters, and tile shapes whose low run spans several box
dimensions.  Tracing confirms which kernel ran (kind 10: micro-op passes)."""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I
from tolerance import TOL, check, energy_tol, grad_tol, state_err

pytestmark = pytest.mark.gpu
MICRO = 10


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def traced_apply(Q, c, s, params):
    import torch
    torch.cuda.synchronize()
    Q.trace_enable(True)
    c.apply(s, params)
    torch.cuda.synchronize()
    _, _, kinds = Q.trace_read()
    Q.trace_enable(False)
    return kinds


@pytest.mark.parametrize("n,opts", [(9, {}), (12, {}), (13, dict(tile_bits=13, low_bits=4)),
                                    (16, dict(tile_bits=13, low_bits=6)), (18, dict(tile_bits=12, low_bits=5)),
                                    (20, {})])
def test_micro_forward_matches_oracle_and_interpreter(Q, n, opts):
    circ = I.random_mixed_circuit(n, 120, seed=4000 + n, max_ctrls=2)
    params = I.uniform_params(circ.n_params, 4100 + n)
    psi0 = I.random_state(n, 4200 + n)
    want = O.evolve(circ, params, psi0)
    c = Q.circuit_from(circ).finalize(Q.C64, fuse=3, **opts)
    s = Q.State(n, Q.C64).set_qs(psi0)
    kinds = traced_apply(Q, c, s, params)
    assert (kinds == MICRO).any(), "no pass ran as micro-ops"
    got = s.get_qs().astype(np.complex128)
    check(f"micro forward n={n} {opts}", state_err(got, want), TOL[0])
    ci = Q.circuit_from(circ).finalize(Q.C64, fuse=2, **opts)
    si = Q.State(n, Q.C64).set_qs(psi0)
    kinds_i = traced_apply(Q, ci, si, params)
    assert not (kinds_i == MICRO).any()
    check(f"interpreter forward n={n} {opts}", state_err(si.get_qs(), want), TOL[0])


def test_micro_random_recipe_20q(Q):
    n = 20
    circ = I.random_circuit(n, 500, seed=2)
    want = O.evolve(circ, [], O.zero_state(n))
    c = Q.circuit_from(circ).finalize(Q.C64, fuse=3)
    s = Q.State(n, Q.C64).set_basis(0)
    kinds = traced_apply(Q, c, s, [])
    assert (kinds == MICRO).all(), kinds
    check("micro random20", state_err(s.get_qs(), want), TOL[0])


@pytest.mark.parametrize("n,opts", [(10, {}), (12, {}), (15, dict(tile_bits=12, low_bits=4)), (17, {})])
def test_micro_adjoint_matches_oracle(Q, n, opts):
    circ = I.random_mixed_circuit(n, 50, seed=4300 + n, max_ctrls=2)
    gates = [I.Gate(g.kind, g.targets, g.ctrls, (g.param % 6) if g.param >= 0 else -1, g.coef, g.const, g.matrix)
             for g in circ.gates]
    circ = I.Circuit(n, gates, 6)
    ham = I.random_pauli_sum(n, 8, seed=4400 + n)
    params = I.uniform_params(6, 4500 + n)
    psi0 = I.random_state(n, 4600 + n)
    E0, g0 = O.adjoint_gradient(circ, ham, params, psi0)
    import torch
    c = Q.circuit_from(circ).finalize(Q.C64, fuse=3, **opts)
    psi, lam = Q.State(n, Q.C64).set_qs(psi0), Q.State(n, Q.C64)
    torch.cuda.synchronize()
    Q.trace_enable(True)
    E, g = Q.expectation_with_grad(psi, lam, c, Q.Hamiltonian(ham), params)
    torch.cuda.synchronize()
    _, _, kinds = Q.trace_read()
    Q.trace_enable(False)
    assert (kinds == MICRO).sum() >= 2
    check(f"micro adjoint n={n} energy", abs(E - E0), energy_tol(0, ham))
    check(f"micro adjoint n={n} grad", np.abs(g - g0), grad_tol(0, ham, circ))
    check(f"micro adjoint n={n} uncomputed psi", state_err(psi.get_qs(), psi0), 2 * TOL[0])
