"""GPU parity of the density-matrix simulator against the FP64 density-matrix
oracle: rho after noisy circuits (every channel kind, custom Kraus included),
tr(rho H), the noiseless case against the state-vector oracle, and a 14-qubit
density matrix (a 28-qubit vector) against the state-vector oracle.
Tolerances: the rule of tests/tolerance.py, rho as a vector of 4^n entries
(its Frobenius norm is that vector's 2-norm), tr(rho) as the energy of H = I."""
import numpy as np
import pytest

from oracle import dm_oracle as D
from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

from tolerance import TOL, check, energy_tol, state_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def _rho(Q, s, n):
    v = s.get_qs().astype(np.complex128)
    return v.reshape(1 << n, 1 << n).T  # vec[x + 2^n y] = rho[x, y]


KINDS = [("pauli", (0.1, 0.05, 0.2)), ("depolarizing", (0.3,)), ("amplitude_damping", (0.4,)),
         ("phase_damping", (0.25,))]


@pytest.mark.parametrize("dt", [0, 1])
def test_noisy_circuit_matches_oracle(Q, dt):
    n = 5
    circ = I.random_mixed_circuit(n, 30, 7, with_matrix=True)
    params = I.uniform_params(circ.n_params, 3)
    ch = {i: [(KINDS[i % 4][0], KINDS[i % 4][1], (3 * i) % n)] for i in range(-1, len(circ.gates), 4)}
    c = Q.dm_circuit_from(circ, ch)
    # a custom Kraus channel (amplitude damping written out) at the end
    g = 0.2
    c.add_channel("kraus", 1, (), kraus=[np.array([[1, 0], [0, np.sqrt(1 - g)]]), np.array([[0, np.sqrt(g)], [0, 0]])])
    c.finalize(dt)
    s = Q.State(2 * n, dt).set_basis(0)
    c.apply(s, params)
    want = D.run(circ, params, ch, n)
    want = D.apply_channel(want, n, D.channel_kraus("amplitude_damping", (g,)), 1)
    check(f"dm noisy rho dt={dt}", state_err(_rho(Q, s, n), want), TOL[dt])
    for seed in range(3):
        ham = I.random_pauli_sum(n, 10, seed)
        E = Q.dm_expectation(s, Q.Hamiltonian(ham))
        check(f"dm noisy energy {seed} dt={dt}", abs(E - D.expectation(want, ham)), energy_tol(dt, ham))


@pytest.mark.parametrize("dt", [0, 1])
def test_noiseless_density_matrix_equals_pure_state(Q, dt):
    n = 6
    circ = I.hea_circuit(n, 3)
    params = I.uniform_params(circ.n_params, 9)
    c = Q.dm_circuit_from(circ).finalize(dt)
    s = Q.State(2 * n, dt).set_basis(0)
    c.apply(s, params)
    psi = O.evolve(circ, params, O.zero_state(n))
    check(f"dm noiseless rho dt={dt}", state_err(_rho(Q, s, n), np.outer(psi, psi.conj())), TOL[dt])
    ham = I.chain_zz_x(n, 0.5)
    check(f"dm noiseless energy dt={dt}", abs(Q.dm_expectation(s, Q.Hamiltonian(ham)) - O.expectation(psi, ham)),
          energy_tol(dt, ham))


def test_density_matrix_14_qubits(Q):
    """A 14-qubit density matrix (2^28 complex64 entries) in the launch
    configuration the benchmark times: without channels tr(rho H) equals the
    state-vector oracle's <psi|H|psi>; with depolarizing noise after every layer
    the trace stays 1 and the energy moves toward 0 (the fully mixed value)."""
    n = 14
    circ = I.hea_circuit(n, 2)
    params = I.uniform_params(circ.n_params, 5)
    ham = I.chain_zz_x(n, 0.5)
    H = Q.Hamiltonian(ham)
    one = Q.Hamiltonian(I.pauli_sum_from_strings(n, [(1.0, "")]))
    s = Q.State(2 * n, Q.C64).set_basis(0)
    Q.dm_circuit_from(circ).finalize(Q.C64).apply(s, params)
    E0 = O.expectation(O.evolve(circ, params, O.zero_state(n)), ham)
    check("dm14 noiseless energy", abs(Q.dm_expectation(s, H) - E0), energy_tol(0, ham))
    layer_end = [i for i, g in enumerate(circ.gates) if g.kind == "X" and g.targets == (n - 1,)]
    ch = {i: [("depolarizing", (0.05,), q) for q in range(n)] for i in layer_end}
    s.set_basis(0)
    Q.dm_circuit_from(circ, ch).finalize(Q.C64).apply(s, params)
    check("dm14 noisy trace", abs(Q.dm_expectation(s, one) - 1.0), TOL[0])
    assert abs(Q.dm_expectation(s, H)) < abs(E0)
