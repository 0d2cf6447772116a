"""GPU parity of Monte-Carlo trajectory noise (§3.3) against the FP64 oracle:
the branch taken at every channel site (bit-exact wherever the oracle's decision
is further than the state's rounding from a branch boundary; always for Pauli
and depolarizing channels, whose weights are constants), the final state of
each trajectory, the trajectory energies, the mean adjoint gradient of
Pauli-channel trajectories, convergence of the mean to tr(rho H), 64-bit
trajectory counters, the largest shared-memory states, and states beyond
shared memory on the fused tile passes.

Tolerances: the rule of tests/tolerance.py (amplitudes tol, energies
tol * max(1, sum |c_k|)); the mean gradients are held to the energy's bound,
tighter than the rule's gradient bound."""
import math

import numpy as np
import pytest

from oracle import dm_oracle as D
from oracle import qsim_oracle as O
from oracle import traj_oracle as T
from paper_2406_17248_gb300 import inputs as I

from tolerance import TOL, check, energy_tol, state_err

pytestmark = pytest.mark.gpu
MARGIN = {0: 1e-5, 1: 1e-12}


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def _kraus3(seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(6, 2)) + 1j * rng.normal(size=(6, 2))
    q, _ = np.linalg.qr(a)
    return [q[2 * i:2 * i + 2, :] for i in range(3)]


def _mixed_noise(n, layers, seed):
    circ = I.hea_circuit(n, layers)
    params = I.uniform_params(circ.n_params, seed)
    kinds = [("depolarizing", (0.2,)), ("amplitude_damping", (0.3,)), ("pauli", (0.1, 0.15, 0.05)),
             ("phase_damping", (0.4,))]
    ch = {-1: [("amplitude_damping", (0.5,), 0)]}
    for i in range(0, len(circ.gates), 2):
        k, p = kinds[(i // 2) % 4]
        ch[i] = [(k, p, (i // 2) % n)]
    ch[len(circ.gates) - 1] = ch.get(len(circ.gates) - 1, []) + [("kraus", (), n - 1, _kraus3(seed))]
    return circ, params, ch


@pytest.mark.parametrize("dt", [0, 1])
def test_states_and_branches_match_oracle(Q, dt):
    n = 5
    circ, params, ch = _mixed_noise(n, 2, 3)
    eng = Q.trajectories_from(circ, ch, dt)
    seed = 2024
    ham = I.chain_zz_x(n, 0.5)
    e, branches = eng.run(Q.Hamiltonian(ham), params, 48, seed, choices=True)
    checked = 0
    for t in range(48):
        psi, choices, margins = T.trajectory(circ, params, ch, seed, t)
        if min(margins) < MARGIN[dt]:
            continue
        checked += 1
        assert list(branches[t]) == choices, t
        s = Q.State(n, dt)
        eng.state(params, seed, t, s)
        check(f"traj {t} state dt={dt}", state_err(s.get_qs(), psi), TOL[dt])
        check(f"traj {t} energy dt={dt}", abs(e[t] - O.expectation(psi, ham)), energy_tol(dt, ham))
    assert checked >= 40


@pytest.mark.parametrize("dt", [0, 1])
def test_pauli_channel_gradients_match_oracle(Q, dt):
    n = 6
    circ = I.hea_circuit(n, 2)
    params = I.uniform_params(circ.n_params, 11)
    ham = I.chain_zz_x(n, 0.7)
    ch = {i: [("depolarizing", (0.1,), i % n), ("pauli", (0.05, 0.02, 0.08), (i + 3) % n)]
          for i in range(0, len(circ.gates), 3)}
    eng = Q.trajectories_from(circ, ch, dt)
    n_t, seed, first = 96, 77, 5
    e, g, branches = eng.run(Q.Hamiltonian(ham), params, n_t, seed, first=first, grad=True, choices=True)
    es, gs = [], []
    for i in range(n_t):
        eo, go, co, _ = T.trajectory_energy_and_grad(circ, ham, params, ch, seed, first + i)
        assert list(branches[i]) == co, i  # constant weights: the same decision on both sides
        es.append(eo)
        gs.append(go)
    tol = energy_tol(dt, ham)
    check(f"traj pauli energies dt={dt}", np.abs(e - np.array(es)), tol)
    check(f"traj pauli mean grad dt={dt}", np.abs(g - np.mean(gs, axis=0)), tol)


def test_gradients_refused_with_damping(Q):
    circ = I.hea_circuit(3, 1)
    eng = Q.trajectories_from(circ, {0: [("amplitude_damping", (0.1,), 0)]}, 0)
    with pytest.raises(Q.QSimError, match="gradients need"):
        eng.run(Q.Hamiltonian(I.chain_zz_x(3)), np.zeros(circ.n_params), 4, 1, grad=True)


def test_mean_converges_to_density_matrix(Q):
    n = 6
    circ = I.hea_circuit(n, 2)
    params = I.uniform_params(circ.n_params, 9)
    ham = I.chain_zz_x(n, 0.5)
    ch = {i: [("depolarizing", (0.05,), i % n), ("amplitude_damping", (0.1,), (i + 2) % n)]
          for i in range(0, len(circ.gates), 3)}
    exact = D.expectation(D.run(circ, params, ch, n), ham)
    eng = Q.trajectories_from(circ, ch, 0)
    e = eng.run(Q.Hamiltonian(ham), params, 20000, seed=31)
    assert abs(e.mean() - exact) < 5 * e.std() / math.sqrt(e.size)
    # and the GPU density-matrix simulator agrees with the exact value
    dmc = Q.dm_circuit_from(circ, ch).finalize(1)
    rho = Q.State(2 * n, 1)
    rho.set_basis(0)
    dmc.apply(rho, params)
    assert Q.dm_expectation(rho, Q.Hamiltonian(ham)) == pytest.approx(exact, abs=1e-10)


def test_zero_noise_is_the_noiseless_state(Q):
    n = 7
    circ = I.hea_circuit(n, 3)
    params = I.uniform_params(circ.n_params, 4)
    ch = {i: [("depolarizing", (0.0,), i % n), ("amplitude_damping", (0.0,), (i + 1) % n)]
          for i in range(0, len(circ.gates), 5)}
    eng = Q.trajectories_from(circ, ch, 1)
    s = Q.State(n, 1)
    eng.state(params, 5, 123, s)
    np.testing.assert_allclose(s.get_qs(), O.evolve(circ, params, O.zero_state(n)), atol=1e-12)


def test_64_bit_trajectory_counters(Q):
    n = 4
    circ = I.hea_circuit(n, 1)
    params = I.uniform_params(circ.n_params, 2)
    ch = {i: [("pauli", (0.2, 0.2, 0.2), i % n)] for i in range(len(circ.gates))}
    eng = Q.trajectories_from(circ, ch, 1)
    first = (1 << 40) + 17
    _, branches = eng.run(Q.Hamiltonian(I.chain_zz_x(n)), params, 16, seed=(1 << 63) + 5, first=first, choices=True)
    for i in range(16):
        assert list(branches[i]) == T.trajectory(circ, params, ch, (1 << 63) + 5, first + i)[1]


@pytest.mark.parametrize("dt,n,grad", [(0, 14, False), (0, 13, True), (1, 13, False), (1, 12, True)])
def test_largest_shared_memory_trajectories(Q, dt, n, grad):
    circ = I.hea_circuit(n, 1)
    params = I.uniform_params(circ.n_params, 6)
    ham = I.chain_zz_x(n, 0.5)
    ch = {i: [("depolarizing", (0.1,), i % n)] for i in range(0, len(circ.gates), 4)}
    eng = Q.trajectories_from(circ, ch, dt)
    info = eng.info()
    assert (info["grid_grad"] if grad else info["grid_energy"]) > 0
    out = eng.run(Q.Hamiltonian(ham), params, 3, seed=8, grad=grad)
    e = out[0] if grad else out
    tol = energy_tol(dt, ham)
    gs = []
    for t in range(3):
        eo, go, _, _ = T.trajectory_energy_and_grad(circ, ham, params, ch, 8, t)
        check(f"traj smem n={n} {t} energy dt={dt}", abs(e[t] - eo), tol)
        gs.append(go)
    if grad:
        check(f"traj smem n={n} mean grad dt={dt}", np.abs(out[1] - np.mean(gs, axis=0)), tol)


@pytest.mark.parametrize("dt", [0, 1])
def test_large_state_trajectories_match_oracle(Q, dt):
    """States beyond one CTA's shared memory run on the fused tile passes: every
    channel kind (the damping / Kraus weights from the qubit's reduced density
    matrix), against the oracle's branches, states and energies."""
    n = 15
    circ, params, ch = _mixed_noise(n, 1, 5)
    eng = Q.trajectories_from(circ, ch, dt)
    assert eng.info()["grid_energy"] == 0
    seed = 99
    ham = I.chain_zz_x(n, 0.5)
    e, branches = eng.run(Q.Hamiltonian(ham), params, 6, seed, first=3, choices=True)
    checked = 0
    for i in range(6):
        psi, choices, margins = T.trajectory(circ, params, ch, seed, 3 + i)
        if min(margins) < MARGIN[dt]:
            continue
        checked += 1
        assert list(branches[i]) == choices, i
        check(f"traj large {i} energy dt={dt}", abs(e[i] - O.expectation(psi, ham)), energy_tol(dt, ham))
        s = Q.State(n, dt)
        eng.state(params, seed, 3 + i, s)
        check(f"traj large {i} state dt={dt}", state_err(s.get_qs(), psi), TOL[dt])
    assert checked >= 4


@pytest.mark.parametrize("dt,n", [(0, 14), (1, 13)])
def test_large_state_pauli_gradients_match_oracle(Q, dt, n):
    """Gradients beyond shared memory (psi and lam do not both fit): each
    trajectory one adjoint evaluation of its circuit on the tile passes, through
    the host and the device-buffer entry points."""
    import torch
    circ = I.hea_circuit(n, 1)
    params = I.uniform_params(circ.n_params, 12)
    ham = I.chain_zz_x(n, 0.6)
    ch = {i: [("depolarizing", (0.15,), i % n), ("pauli", (0.05, 0.1, 0.02), (i + 5) % n)]
          for i in range(0, len(circ.gates), 4)}
    eng = Q.trajectories_from(circ, ch, dt)
    assert eng.info()["grid_grad"] == 0
    n_t, seed = 4, 41
    e, g, branches = eng.run(Q.Hamiltonian(ham), params, n_t, seed, first=2, grad=True, choices=True)
    es, gs = [], []
    for i in range(n_t):
        eo, go, co, _ = T.trajectory_energy_and_grad(circ, ham, params, ch, seed, 2 + i)
        assert list(branches[i]) == co, i
        es.append(eo)
        gs.append(go)
    tol = energy_tol(dt, ham)
    check(f"traj large grad n={n} energies dt={dt}", np.abs(e - np.array(es)), tol)
    check(f"traj large grad n={n} mean grad dt={dt}", np.abs(g - np.mean(gs, axis=0)), tol)
    d_p = torch.tensor(params, dtype=torch.float64, device="cuda")
    d_e = torch.zeros(n_t, dtype=torch.float64, device="cuda")
    d_g = torch.zeros(circ.n_params, dtype=torch.float64, device="cuda")
    eng.run_device(Q.Hamiltonian(ham), d_p, n_t, seed, d_e, d_g, first=2)
    check(f"traj large grad n={n} device energies dt={dt}", np.abs(d_e.cpu().numpy() - np.array(es)), tol)
    check(f"traj large grad n={n} device mean grad dt={dt}", np.abs(d_g.cpu().numpy() - np.mean(gs, axis=0)), tol)
