"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: one rule for every result, tol times the largest magnitude the
result can take (``tolerance.py``): amplitudes tol (1e-11 complex128, 5e-5
complex64), energies tol * max(1, sum |c_k|), gradients that bound times the sum
of |coef| over the gates sharing the parameter, states returned to their start
2 tol.  Each check records its measured error."""
import json
import math
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


def run_circuit(Q, circ, params, dt, psi0=None, **opts):
    c = Q.circuit_from(circ).finalize(dt, **opts)
    s = Q.State(circ.n_qubits, dt)
    if psi0 is None:
        s.set_basis(0)
    else:
        s.set_qs(psi0)
    c.apply(s, params)
    return s.get_qs().astype(np.complex128), c


PLAN_OPTS = [dict(), dict(tile_bits=6, low_bits=1), dict(tile_bits=6, low_bits=3), dict(tile_bits=8, low_bits=2),
             dict(tile_bits=13, low_bits=5), dict(fuse=-1)]


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 10, 13])
def test_apply_mixed_circuits(Q, dt, n):
    circ = I.random_mixed_circuit(n, 60, seed=1000 + n)
    params = I.uniform_params(circ.n_params, 2000 + n)
    psi0 = I.random_state(n, 3000 + n)
    want = O.evolve(circ, params, psi0)
    for opts in PLAN_OPTS:
        got, _ = run_circuit(Q, circ, params, dt, psi0, **opts)
        check(f"apply_mixed n={n} dt={dt} {opts}", state_err(got, want), TOL[dt])


@pytest.mark.parametrize("dt", [0, 1])
def test_random_circuit_recipe_at_20_qubits(Q, dt):
    """The 28-qubit benchmark recipe (500 gates over {H,RX,RY,RZ,CNOT,CZ}) at 20
    qubits, where the oracle runs in seconds; spans many tiles and passes."""
    n = 20
    circ = I.random_circuit(n, 500, seed=2)
    want = O.evolve(circ, [], O.zero_state(n))
    got, c = run_circuit(Q, circ, [], dt)
    check(f"random20 dt={dt}", state_err(got, want), TOL[dt])
    assert c.info()["passes"] < 500 / 4


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [1, 5, 9, 14])
def test_expectation_apply_hamiltonian_inner(Q, dt, n):
    ham = I.random_pauli_sum(n, 15, seed=n)
    a = I.random_state(n, 10 + n)
    b = I.random_state(n, 20 + n)
    H = Q.Hamiltonian(ham)
    sa = Q.State(n, dt).set_qs(a)
    sb = Q.State(n, dt).set_qs(b)
    e = Q.expectation(sa, H)
    tag = f"expectation n={n} dt={dt}"
    check(tag, abs(e - O.expectation(a, ham)), energy_tol(dt, ham))
    Q.apply_hamiltonian(sb, sa, H)
    got = sb.get_qs().astype(np.complex128)
    # ||H psi|| <= sum |c_k|: the amplitudes of lam = H psi carry the energy's bound
    check(tag + " H psi", state_err(got, O.apply_hamiltonian(a, ham)), energy_tol(dt, ham))
    sb.set_qs(b)
    ip = Q.inner_product(sa, sb)
    check(tag + " inner product", abs(ip - O.inner_product(a, b)), TOL[dt])
    check(tag + " norm", abs(sa.norm2() - 1.0), 2 * TOL[dt] + TOL[dt] ** 2)


@pytest.mark.parametrize("dt", [0, 1])
def test_paper_printed_values_through_the_abi(Q, dt):
    g = json.load(open(os.path.join(GOLD, "paper_prints.json")))
    c = Q.Circuit(2).add("RX", [0], const=g["zz_after_rx"]["theta"])
    s = Q.State(2, dt).set_basis(0)
    c.apply(s)
    H = Q.Hamiltonian(I.pauli_sum_from_strings(2, [(1.0, "Z0 Z1")]))
    check(f"paper ZZ after RX dt={dt}", abs(Q.expectation(s, H) - g["zz_after_rx"]["value"]), TOL[dt])
    phi = Q.State(2, dt).set_basis(0)
    Q.Circuit(2).add("RY", [0], const=g["inner_product"]["ry"]).apply(phi)
    ip = Q.inner_product(phi, s)
    check(f"paper inner product dt={dt}", abs(ip - complex(g["inner_product"]["re"], g["inner_product"]["im"])),
          TOL[dt])
    # apply_hamiltonian(X0 Y1) on |00>, then H(0), X(1 <- 0)
    src = Q.State(2, dt).set_basis(0)
    dst = Q.State(2, dt)
    Q.apply_hamiltonian(dst, src, Q.Hamiltonian(I.pauli_sum_from_strings(2, [(1.0, "X0 Y1")])))
    Q.Circuit(2).add("H", [0]).add("X", [1], [0]).apply(dst)
    want = np.array(g["apply_hamiltonian_then_circuit"]["amplitudes_re"]) + \
        1j * np.array(g["apply_hamiltonian_then_circuit"]["amplitudes_im"])
    check(f"paper apply_hamiltonian then circuit dt={dt}", state_err(dst.get_qs(), want), TOL[dt])


@pytest.mark.parametrize("dt", [0, 1])
def test_bell_ghz_closed_forms(Q, dt):
    for n in (2, 3, 8, 17):
        c = Q.Circuit(n).add("H", [0])
        for q in range(1, n):
            c.add("X", [q], [q - 1])
        s = Q.State(n, dt).set_basis(0)
        c.apply(s)
        got = s.get_qs()
        want = np.zeros(1 << n)
        want[0] = want[-1] = 1 / math.sqrt(2)
        check(f"ghz n={n} dt={dt}", state_err(got, want), TOL[dt])


@pytest.mark.parametrize("dt", [0, 1])
def test_adjoint_hea_12q(Q, dt):
    """The 12-qubit HEA workload: 4 layers, 96 parameters U[-pi, pi] (seed 1),
    H = sum Z_i Z_{i+1} + 0.5 sum X_i."""
    n = 12
    circ = I.hea_circuit(n, 4)
    ham = I.chain_zz_x(n)
    params = I.uniform_params(circ.n_params, 1)
    E0, g0 = O.adjoint_gradient(circ, ham, params, O.zero_state(n))
    c = Q.circuit_from(circ).finalize(dt)
    psi, lam = Q.State(n, dt).set_basis(0), Q.State(n, dt)
    E, g = Q.expectation_with_grad(psi, lam, c, Q.Hamiltonian(ham), params)
    check(f"hea12 energy dt={dt}", abs(E - E0), energy_tol(dt, ham))
    check(f"hea12 grad dt={dt}", np.abs(g - g0), grad_tol(dt, ham, circ))
    # psi is returned to the initial state (forward and reverse sweeps: 2 tol)
    check(f"hea12 uncomputed psi dt={dt}", state_err(psi.get_qs(), O.zero_state(n)), 2 * TOL[dt])


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,opts", [(4, {}), (6, dict(tile_bits=6, low_bits=2)), (9, dict(tile_bits=7, low_bits=3)),
                                    (11, {}), (14, dict(tile_bits=10, low_bits=4))])
def test_adjoint_mixed_circuits(Q, dt, n, opts):
    circ = I.random_mixed_circuit(n, 40, seed=500 + n)
    # fold parameters onto 5 shared ones
    gates = [I.Gate(g.kind, g.targets, g.ctrls, (g.param % 5) if g.param >= 0 else -1, g.coef, g.const, g.matrix)
             for g in circ.gates]
    circ = I.Circuit(n, gates, 5)
    ham = I.random_pauli_sum(n, 8, seed=600 + n)
    params = I.uniform_params(5, 700 + n)
    psi0 = I.random_state(n, 800 + n)
    E0, g0 = O.adjoint_gradient(circ, ham, params, psi0)
    c = Q.circuit_from(circ).finalize(dt, **opts)
    psi, lam = Q.State(n, dt).set_qs(psi0), Q.State(n, dt)
    E, g = Q.expectation_with_grad(psi, lam, c, Q.Hamiltonian(ham), params)
    check(f"adjoint_mixed n={n} dt={dt} energy", abs(E - E0), energy_tol(dt, ham))
    check(f"adjoint_mixed n={n} dt={dt} grad", np.abs(g - g0), grad_tol(dt, ham, circ))


@pytest.mark.parametrize("dt", [0, 1])
def test_qaoa_qupack_k5_pin(Q, dt):
    g = json.load(open(os.path.join(GOLD, "qupack_qaoa_k5.json")))
    n, p = g["n_qubits"], g["depth"]
    q = Q.QAOA(n, I.complete_graph(n), p, gamma_scale=1.0, dtype=dt)
    psi, lam = Q.State(n, dt), Q.State(n, dt)
    E, dg, db = q.expectation_with_grad(psi, lam, [g["gamma"]] * p, [g["beta"]] * p)
    te, tg, tb = qaoa_grad_tols(dt, n, 10, 1.0)  # K5: 10 edges, QuPack scaling exp(-i gamma C)
    check(f"qupack_k5 energy dt={dt}", abs(E - g["expectation"]), te)
    check(f"qupack_k5 dgamma dt={dt}", np.abs(dg - g["gamma_grad"]), tg)
    check(f"qupack_k5 dbeta dt={dt}", np.abs(db - g["beta_grad"]), tb)
    check(f"qupack_k5 energy-only dt={dt}",
          abs(q.expectation(psi, [g["gamma"]] * p, [g["beta"]] * p) - g["expectation"]), te)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,p,opts", [(6, 1, {}), (8, 3, dict(tile_bits=6, low_bits=2)), (12, 8, {}),
                                      (14, 4, dict(tile_bits=8, low_bits=3)), (16, 8, dict(tile_bits=12, low_bits=4)),
                                      (18, 2, dict(tile_bits=13))])
def test_qaoa_random_regular(Q, dt, n, p, opts):
    edges = I.random_regular_graph(n, 3, seed=n)
    angles = I.uniform_params(2 * p, n, 0.0, np.pi)
    E0, dg0, db0 = O.qaoa_expectation_with_grad(n, edges, angles[:p], angles[p:], 0.5)
    q = Q.QAOA(n, edges, p, gamma_scale=0.5, dtype=dt, **opts)
    psi, lam = Q.State(n, dt), Q.State(n, dt)
    E, dg, db = q.expectation_with_grad(psi, lam, angles[:p], angles[p:])
    te, tg, tb = qaoa_grad_tols(dt, n, len(edges), 0.5)
    tag = f"qaoa n={n} p={p} dt={dt}"
    check(tag + " energy", abs(E - E0), te)
    check(tag + " dgamma", np.abs(dg - dg0), tg)
    check(tag + " dbeta", np.abs(db - db0), tb)
    # energy-only and evolve paths
    check(tag + " energy-only", abs(q.expectation(psi, angles[:p], angles[p:]) - E0), te)
    want = O.qaoa_layers_state(n, edges, angles[:p], angles[p:], 0.5)
    check(tag + " state", state_err(psi.get_qs(), want), TOL[dt])


def test_qaoa_24q_against_stored_oracle_values(Q):
    path = os.path.join(GOLD, "qaoa24_p8.json")
    g = json.load(open(path))
    n, p = g["n"], g["p"]
    edges = [tuple(e) for e in g["edges"]]
    assert edges == I.random_regular_graph(n, 3, g["seed"])
    for dt in (0, 1):
        q = Q.QAOA(n, edges, p, gamma_scale=g["gamma_scale"], dtype=dt)
        psi, lam = Q.State(n, dt), Q.State(n, dt)
        E, dg, db = q.expectation_with_grad(psi, lam, g["gamma"], g["beta"])
        te, tg, tb = qaoa_grad_tols(dt, n, len(edges), g["gamma_scale"])
        check(f"qaoa24 stored energy dt={dt}", abs(E - g["energy"]), te)
        check(f"qaoa24 stored dgamma dt={dt}", np.abs(np.array(dg) - g["dgamma"]), tg)
        check(f"qaoa24 stored dbeta dt={dt}", np.abs(np.array(db) - g["dbeta"]), tb)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [3, 10, 16])
def test_sampling_matches_oracle_on_the_same_state(Q, dt, n):
    circ = I.random_circuit(n, 8 * n, seed=40 + n)
    s = Q.State(n, dt).set_basis(0)
    Q.circuit_from(circ).apply(s)
    shots, seed = 20000, 12345 + n
    got = Q.sample(s, shots, seed)
    amps = s.get_qs().astype(np.complex128)
    want = O.sample(amps, shots, seed)
    bad = np.nonzero(got != want)[0]
    # a mismatch is allowed only where the uniform sits within rounding of a CDF step
    p = amps.real ** 2 + amps.imag ** 2
    cdf = np.cumsum(p)
    for sidx in bad:
        u = O.shot_uniform(seed, int(sidx)) * cdf[-1]
        assert np.min(np.abs(cdf - u)) < 1e-12, (sidx, got[sidx], want[sidx])
    assert len(bad) <= 2


def test_error_paths(Q):
    s = Q.State(4, 0)
    h = Q.Hamiltonian(I.pauli_sum_from_strings(5, [(1.0, "Z0")]))
    with pytest.raises(Q.QSimError, match="qubit count"):
        Q.expectation(s, h)
    c = Q.circuit_from(I.hea_circuit(4, 1)).finalize(0)
    with pytest.raises(Q.QSimError, match="different states"):
        Q.expectation_with_grad(s, s, c, Q.Hamiltonian(I.chain_zz_x(4)), np.zeros(8))
    with pytest.raises(Q.QSimError, match="too few parameters"):
        c.apply(s, np.zeros(3))
    with pytest.raises(Q.QSimError, match="basis index"):
        s.set_basis(16)
    q = Q.QAOA(5, [(0, 1)], 2)
    with pytest.raises(Q.QSimError, match="n/dtype"):
        q.expectation(s, [0, 0], [0, 0])


@pytest.mark.parametrize("dt", [0, 1])
def test_gradient_for_a_list_of_hamiltonians(Q, dt):
    """§4.1: energies [n_ham] and gradients [n_ham, n_params] in one call against
    the oracle's adjoint gradient per Hamiltonian."""
    n = 9
    circ = I.random_mixed_circuit(n, 40, 17, with_matrix=False)
    params = I.uniform_params(circ.n_params, 5)
    hams = [I.chain_zz_x(n, 0.5), I.random_pauli_sum(n, 12, 3), I.pauli_sum_from_strings(n, [(1.0, "Z0")])]
    psi, lam = Q.State(n, dt).set_basis(0), Q.State(n, dt)
    c = Q.circuit_from(circ).finalize(dt)
    E, G = Q.expectation_with_grad_multi(psi, lam, c, [Q.Hamiltonian(h) for h in hams], params)
    assert G.shape == (3, circ.n_params)
    for k, h in enumerate(hams):
        E0, G0 = O.adjoint_gradient(circ, h, params, O.zero_state(n))
        check(f"multi-ham {k} energy dt={dt}", abs(E[k] - E0), energy_tol(dt, h))
        check(f"multi-ham {k} grad dt={dt}", np.abs(G[k] - G0), grad_tol(dt, h, circ))
    # psi is back at |0...0> afterwards (up to rounding)
    assert abs(abs(complex(psi.amplitudes[0].item())) - 1.0) <= 1e-4


@pytest.mark.parametrize("dt", [0, 1])
def test_measurement_collapse_matches_oracle(Q, dt):
    """Mid-circuit measurement: the outcome (decided in FP64 on both sides; cases
    within 1e-9 of the decision boundary are skipped) and the collapsed state."""
    n = 10
    checked = 0
    for seed in range(12):
        psi0 = I.random_state(n, 100 + seed)
        q = seed % n
        base = psi0.astype(np.complex64 if dt == 0 else np.complex128).astype(np.complex128)
        o_or, st_or, p1 = O.measure(base, n, q, seed)
        u = O.shot_uniform(seed, 0)
        if abs((1 - p1) - u) < 1e-9:
            continue
        s = Q.State(n, dt).set_qs(psi0)
        o = Q.measure(s, q, seed)
        assert o == o_or
        check(f"measure collapse seed={seed} dt={dt}", state_err(s.get_qs(), st_or), TOL[dt])
        checked += 1
    assert checked >= 10


@pytest.mark.parametrize("dt", [0, 1])
def test_autotuned_plan_stays_exact(Q, dt):
    """The autotuner (timing of candidate tile shapes) keeps a plan whose results
    still match the oracle, amplitudes and adjoint gradients."""
    n = 14
    circ = I.random_mixed_circuit(n, 60, 23, with_matrix=False)
    params = I.uniform_params(circ.n_params, 8)
    c = Q.circuit_from(circ).finalize(dt)
    scratch = Q.State(n, dt).set_basis(0)
    best = c.autotune(scratch, params, reps=1)
    assert best["ms"] > 0 and 6 <= best["tile_bits"] <= 13 and 2 <= best["low_bits"] <= 5
    psi0 = I.random_state(n, 4)
    s = Q.State(n, dt).set_qs(psi0)
    c.apply(s, params)
    want = O.evolve(circ, params, psi0)
    check(f"autotuned state dt={dt}", state_err(s.get_qs(), want), TOL[dt])
    ham = I.chain_zz_x(n, 0.5)
    psi, lam = Q.State(n, dt).set_basis(0), Q.State(n, dt)
    E, G = Q.expectation_with_grad(psi, lam, c, Q.Hamiltonian(ham), params)
    E0, G0 = O.adjoint_gradient(circ, ham, params, O.zero_state(n))
    check(f"autotuned energy dt={dt}", abs(E - E0), energy_tol(dt, ham))
    check(f"autotuned grad dt={dt}", np.abs(G - G0), grad_tol(dt, ham, circ))


@pytest.mark.parametrize("dt", [0, 1])
def test_qaoa_one_shot_call_reproduces_printed_qupack_values(Q, dt):
    """qs_qaoa_evaluate (no handles, the shape of the QuPack call of §6.2) on the
    paper's K5 depth-10 example: the printed expectation and 20 gradients."""
    g = json.load(open(os.path.join(GOLD, "qupack_qaoa_k5.json")))
    n, p = g["n_qubits"], g["depth"]
    E, dg, db = Q.qaoa_evaluate(n, I.complete_graph(n), p, [g["gamma"]] * p, [g["beta"]] * p, 1.0, dt)
    te, tg, tb = qaoa_grad_tols(dt, n, 10, 1.0)
    check(f"qaoa_evaluate k5 energy dt={dt}", abs(E - g["expectation"]), te)
    check(f"qaoa_evaluate k5 dgamma dt={dt}", np.abs(dg - np.array(g["gamma_grad"])), tg)
    check(f"qaoa_evaluate k5 dbeta dt={dt}", np.abs(db - np.array(g["beta_grad"])), tb)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n_ctrl", [7, 8, 9])
def test_many_controls_per_gate_kernels(Q, dt, n_ctrl):
    """Single-gate kernels at the edge of their fixed-bit table (target +
    controls <= 8 bits take the fast kernels, more fall back to the generic
    ones): multi-controlled X, RY and phase gates on qubit 0 and qubit 11."""
    n = 12
    rng = np.random.default_rng(n_ctrl)
    gates = [I.Gate("H", (q,)) for q in range(n)]
    for t in (0, 11):
        ctrls = tuple(int(c) for c in rng.choice([q for q in range(n) if q != t], n_ctrl, replace=False))
        gates += [I.Gate("X", (t,), ctrls), I.Gate("RY", (t,), ctrls, const=0.7), I.Gate("PS", (t,), ctrls, const=1.1),
                  I.Gate("RZ", (t,), ctrls, const=-0.4)]
    circ = I.Circuit(n, gates)
    want = O.evolve(circ, [], O.zero_state(n))
    got, _ = run_circuit(Q, circ, [], dt, fuse=-1)
    check(f"many controls {n_ctrl} dt={dt}", state_err(got, want), TOL[dt])


def test_c128_exact_forms_per_gate(Q):
    """Complex128 gates whose entries are 0, +-1, +-i (X, Y, Z, S, SDG and their
    controlled forms: swaps and sign flips only) and the Hadamard form, through
    the per-gate kernels, against the oracle on a random state."""
    n = 11
    rng = np.random.default_rng(5)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    gates = []
    for kind in ("X", "Y", "Z", "S", "SDG", "H"):
        for t in (0, 1, 6, 10):
            gates.append(I.Gate(kind, (t,)))
            c = (t + 3) % n
            gates.append(I.Gate(kind, (t,), (c,)))
            gates.append(I.Gate(kind, (t,), (c, (t + 5) % n)))
    circ = I.Circuit(n, gates)
    want = O.evolve(circ, [], psi0)
    got, _ = run_circuit(Q, circ, [], 1, psi0=psi0, fuse=-1)
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("opts", PLAN_OPTS[:5])
def test_c128_real_and_unit_ops_fused(Q, opts):
    """Complex128 tile passes with the real-matrix op (H, RY, X, Z runs) and the
    unit-diagonal op (Z, S, SDG runs, CZ, controlled S), including diagonal and
    control qubits outside the tile, against the oracle."""
    n = 14
    rng = np.random.default_rng(9)
    psi0 = I.random_state(n, 77)
    gates = []
    for _ in range(120):
        t = int(rng.integers(n))
        r = rng.random()
        if r < 0.25:  # a run of real one-qubit gates on t
            for k in rng.choice(["H", "RY", "X", "Z"], 3):
                gates.append(I.Gate(str(k), (t,), const=float(rng.uniform(-3, 3)) if k == "RY" else 0.0))
        elif r < 0.45:  # a run of unit diagonals on t
            for k in rng.choice(["Z", "S", "SDG"], 3):
                gates.append(I.Gate(str(k), (t,)))
        else:
            c = int((t + 1 + rng.integers(n - 1)) % n)
            k = str(rng.choice(["H", "RY", "Z", "S", "SDG", "X", "RX"]))
            gates.append(I.Gate(k, (t,), (c,), const=float(rng.uniform(-3, 3)) if k in ("RY", "RX") else 0.0))
    circ = I.Circuit(n, gates)
    want = O.evolve(circ, [], psi0)
    got, _ = run_circuit(Q, circ, [], 1, psi0, **opts)
    check(f"c128 real/unit fused {opts}", state_err(got, want), TOL[1])


@pytest.mark.parametrize("n,p,tb,lb,gs", [(14, 2, 9, 2, 0.5), (15, 3, 9, 3, 1.0), (16, 3, 10, 3, 0.5),
                                          (18, 4, 11, 3, 0.5), (20, 8, 12, 3, 0.5), (21, 2, 12, 3, 1.0)])
def test_qaoa_two_shape_passes(Q, n, p, tb, lb, gs):
    """The complex64 passes with separate forward and reverse tile shapes (the
    engine bench.py times at 30 qubits), forced with small tiles so that many
    tiles and passes run: energy, gradients and the evolved state against the
    oracle."""
    edges = I.random_regular_graph(n, 3 if n % 2 == 0 else 4, seed=n)
    ang = I.uniform_params(2 * p, n + 1, 0.0, np.pi)
    E0, dg0, db0 = O.qaoa_expectation_with_grad(n, edges, ang[:p], ang[p:], gs)
    q = Q.QAOA(n, edges, p, gamma_scale=gs, dtype=0, tile_bits=tb, low_bits=lb, engine=2)
    psi, lam = Q.State(n, 0), Q.State(n, 0)
    E, dg, db = q.expectation_with_grad(psi, lam, ang[:p], ang[p:])
    te, tg, tb_ = qaoa_grad_tols(0, n, len(edges), gs)
    tag = f"qaoa two-shape n={n} p={p}"
    check(tag + " energy", abs(E - E0), te)
    check(tag + " dgamma", np.abs(dg - dg0), tg)
    check(tag + " dbeta", np.abs(db - db0), tb_)
    check(tag + " energy-only", abs(q.expectation(psi, ang[:p], ang[p:]) - E0), te)
    want = O.qaoa_layers_state(n, edges, ang[:p], ang[p:], gs)
    check(tag + " state", state_err(psi.get_qs(), want), TOL[0])
    # max cut from the lazily built cut-value array
    assert q.max_cut() == O.maxcut_brute_force(n, edges)


@pytest.mark.parametrize("beta", [(0.3, 0.5, 1.0), (2.9, 0.5, 1.0), (2.9, 3.0, 0.2), (2.5, 2.8, -2.9)])
def test_qaoa_scaled_mixer_forms_and_flip(Q, beta):
    """The two-shape passes apply RX as [[1, -it], [-it, 1]] in one of two forms
    (t = s/c, or t = -c/s with the qubits flipped in the data): angles with
    zero to three layers in the flipped form, so the energy plan ends flipped or
    not; energy, gradients and the evolved state against the oracle."""
    n, p, gs = 18, 3, 0.5
    edges = I.random_regular_graph(n, 3, seed=11)
    gamma = np.array([0.4, 1.1, 2.3])
    beta = np.array(beta)
    E0, dg0, db0 = O.qaoa_expectation_with_grad(n, edges, gamma, beta, gs)
    q = Q.QAOA(n, edges, p, gamma_scale=gs, dtype=0, tile_bits=11, low_bits=3, engine=2)
    psi, lam = Q.State(n, 0), Q.State(n, 0)
    E, dg, db = q.expectation_with_grad(psi, lam, gamma, beta)
    te, tg, tb_ = qaoa_grad_tols(0, n, len(edges), gs)
    tag = f"qaoa scaled mixer beta={tuple(beta)}"
    check(tag + " energy", abs(E - E0), te)
    check(tag + " dgamma", np.abs(dg - dg0), tg)
    check(tag + " dbeta", np.abs(db - db0), tb_)
    check(tag + " energy-only", abs(q.expectation(psi, gamma, beta) - E0), te)
    want = O.qaoa_layers_state(n, edges, gamma, beta, gs)
    check(tag + " state", state_err(psi.get_qs(), want), TOL[0])
