"""GPU parity of the per-circuit micro-op kernels (option fuse = 4, compiled at
finalize by the runtime compiler) against the FP64 oracle and against the
library's micro-op kernels (fuse = 3).  The generated kernels run the same op
bodies on the same tiles in the same order, with the op dispatch taken out, so
their states, energies and gradients are expected to equal the library
kernels' bit for bit.  Tracing confirms which kernel ran (kind 11: generated
passes; kind 10: the library's micro-op passes)."""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I
from tolerance import TOL, check, energy_tol, grad_tol, state_err

pytestmark = pytest.mark.gpu
MICRO, GEN = 10, 11


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def traced(Q, fn):
    import torch
    torch.cuda.synchronize()
    Q.trace_enable(True)
    out = fn()
    torch.cuda.synchronize()
    _, _, kinds = Q.trace_read()
    Q.trace_enable(False)
    return out, kinds


@pytest.mark.parametrize("n,opts", [(12, {}), (16, dict(tile_bits=13, low_bits=6)), (18, dict(tile_bits=12, low_bits=5)),
                                    (20, {})])
def test_generated_forward_equals_micro_and_matches_oracle(Q, n, opts):
    circ = I.random_mixed_circuit(n, 120, seed=5000 + n, max_ctrls=2)
    params = I.uniform_params(circ.n_params, 5100 + n)
    psi0 = I.random_state(n, 5200 + n)
    want = O.evolve(circ, params, psi0)
    cg = Q.circuit_from(circ).finalize(Q.C64, fuse=4, **opts)
    sg = Q.State(n, Q.C64).set_qs(psi0)
    _, kinds = traced(Q, lambda: cg.apply(sg, params))
    assert (kinds == GEN).any() and not (kinds == MICRO).any(), kinds
    got = sg.get_qs()
    check(f"generated forward n={n} {opts}", state_err(got.astype(np.complex128), want), TOL[0])
    cm = Q.circuit_from(circ).finalize(Q.C64, fuse=3, **opts)
    sm = Q.State(n, Q.C64).set_qs(psi0)
    cm.apply(sm, params)
    ref = sm.get_qs()
    assert np.array_equal(got.view(np.float32), ref.view(np.float32)), \
        f"generated and library micro-op passes differ: max {np.abs(got - ref).max():.3e}"


def test_generated_random_recipe_22q(Q):
    n = 22
    circ = I.random_circuit(n, 500, seed=2)
    want = O.evolve(circ, [], O.zero_state(n))
    cg = Q.circuit_from(circ).finalize(Q.C64, fuse=4)
    s = Q.State(n, Q.C64).set_basis(0)
    _, kinds = traced(Q, lambda: cg.apply(s, []))
    assert (kinds == GEN).all(), kinds
    got = s.get_qs()
    check("generated random22", state_err(got.astype(np.complex128), want), TOL[0])
    cm = Q.circuit_from(circ).finalize(Q.C64, fuse=3)
    sm = Q.State(n, Q.C64).set_basis(0)
    cm.apply(sm, [])
    assert np.array_equal(got.view(np.float32), sm.get_qs().view(np.float32))


@pytest.mark.parametrize("n,opts", [(12, {}), (15, dict(tile_bits=12, low_bits=4)), (17, {})])
def test_generated_adjoint_equals_micro_and_matches_oracle(Q, n, opts):
    circ = I.random_mixed_circuit(n, 50, seed=5300 + n, max_ctrls=2)
    gates = [I.Gate(g.kind, g.targets, g.ctrls, (g.param % 6) if g.param >= 0 else -1, g.coef, g.const, g.matrix)
             for g in circ.gates]
    circ = I.Circuit(n, gates, 6)
    ham = I.random_pauli_sum(n, 8, seed=5400 + n)
    H = Q.Hamiltonian(ham)
    params = I.uniform_params(6, 5500 + n)
    psi0 = I.random_state(n, 5600 + n)
    E0, g0 = O.adjoint_gradient(circ, ham, params, psi0)
    res = {}
    for fuse in (4, 3):
        c = Q.circuit_from(circ).finalize(Q.C64, fuse=fuse, **opts)
        psi, lam = Q.State(n, Q.C64).set_qs(psi0), Q.State(n, Q.C64)
        (E, g), kinds = traced(Q, lambda: Q.expectation_with_grad(psi, lam, c, H, params))
        assert (kinds == (GEN if fuse == 4 else MICRO)).sum() >= 2, kinds
        res[fuse] = (E, np.asarray(g), psi.get_qs())
    E, g, psi_u = res[4]
    check(f"generated adjoint n={n} energy", abs(E - E0), energy_tol(0, ham))
    check(f"generated adjoint n={n} grad", np.abs(g - g0), grad_tol(0, ham, circ))
    check(f"generated adjoint n={n} uncomputed psi", state_err(psi_u.astype(np.complex128), psi0), 2 * TOL[0])
    assert E == res[3][0] and np.array_equal(g, res[3][1])
    assert np.array_equal(psi_u.view(np.float32), res[3][2].view(np.float32))


def test_generated_kernels_are_cached_by_source(Q):
    import time
    n = 20
    circ = I.random_circuit(n, 300, seed=7)
    t0 = time.perf_counter()
    Q.circuit_from(circ).finalize(Q.C64, fuse=4)
    first = time.perf_counter() - t0
    t0 = time.perf_counter()
    c2 = Q.circuit_from(circ).finalize(Q.C64, fuse=4)
    second = time.perf_counter() - t0
    s = Q.State(n, Q.C64).set_basis(0)
    _, kinds = traced(Q, lambda: c2.apply(s, []))
    assert (kinds == GEN).all()
    assert second < 0.5 * first, (first, second)


def test_default_compiles_passes_within_budget_22q(Q):
    """fuse = 1 from 22 qubits: passes within the op budget compiled for the
    circuit, larger ones (the first adjoint pass of this ansatz, 131 ops) on the
    library kernel; all results equal fuse = 3's bit for bit."""
    n = 22
    circ = I.hea_circuit(n, 4)
    rng = np.random.default_rng(5700)
    ham = I.tfim(n, rng)
    H = Q.Hamiltonian(ham)
    params = rng.uniform(-np.pi, np.pi, circ.n_params)
    res = {}
    for fuse in (1, 3):
        c = Q.circuit_from(circ).finalize(Q.C64, fuse=fuse)
        psi, lam = Q.State(n, Q.C64).set_basis(0), Q.State(n, Q.C64)
        (E, g), kinds = traced(Q, lambda: Q.expectation_with_grad(psi, lam, c, H, params))
        res[fuse] = (E, np.asarray(g), kinds)
    kinds = res[1][2]
    assert (kinds == GEN).any() and (kinds == MICRO).sum() == 1, kinds
    assert not (res[3][2] == GEN).any()
    assert res[1][0] == res[3][0] and np.array_equal(res[1][1], res[3][1])
    E0, g0 = O.adjoint_gradient(circ, ham, params, O.zero_state(n))
    check("default 22q HEA energy", abs(res[1][0] - E0), energy_tol(0, ham))
    check("default 22q HEA grad", np.abs(res[1][1] - g0), grad_tol(0, ham, circ))
