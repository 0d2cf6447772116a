"""Parity at the benchmark sizes, in the launch configuration bench.py times,
where the oracle cannot simulate the whole problem: exact results that hold at
any size (the depth-1 QAOA closed form, itself pinned against the oracle),
symmetries of the QAOA energy, a circuit followed by its inverse, and sampled
instances of the batched workload checked one by one against the oracle.
Tolerances: the rule of tests/tolerance.py."""
import math

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

from tolerance import TOL, check, energy_tol, grad_tol, qaoa_grad_tols

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


def _bench_graph(n=30, seed=3):
    return I.random_regular_graph(n, 3, seed)


def test_qaoa30_depth1_against_closed_form(Q):
    """30 qubits, complex64, the benchmark graph, p = 1, RZZ(gamma) per edge:
    energy against the closed form and gradients against its central
    differences (the formula is smooth; h = 1e-5 in float64)."""
    n, edges = 30, _bench_graph()
    q = Q.QAOA(n, edges, 1, 0.5, Q.C64)
    psi, lam = Q.State(n, Q.C64), Q.State(n, Q.C64)
    te, tg, tb = qaoa_grad_tols(0, n, len(edges), 0.5)
    for g, b in [(0.61, 0.37), (-1.3, 2.2), (2.9, -0.8)]:
        E, dg, db = q.expectation_with_grad(psi, lam, [g], [b])
        Ec = O.qaoa_p1_energy_closed_form(n, edges, g, b, 0.5)
        h = 1e-5
        dgc = (O.qaoa_p1_energy_closed_form(n, edges, g + h, b, 0.5) -
               O.qaoa_p1_energy_closed_form(n, edges, g - h, b, 0.5)) / (2 * h)
        dbc = (O.qaoa_p1_energy_closed_form(n, edges, g, b + h, 0.5) -
               O.qaoa_p1_energy_closed_form(n, edges, g, b - h, 0.5)) / (2 * h)
        check(f"qaoa30 p1 energy ({g}, {b})", abs(E - Ec), te)
        check(f"qaoa30 p1 dgamma ({g}, {b})", abs(dg[0] - dgc), tg)
        check(f"qaoa30 p1 dbeta ({g}, {b})", abs(db[0] - dbc), tb)


def test_qaoa30_depth8_symmetries_and_determinism(Q):
    """The benchmark workload (p = 8, angles U[0, pi] seed 3): E(-theta) = E(theta)
    with negated gradients (complex conjugation of a real-start circuit);
    shifting one mixer angle by 2 pi (RX(b + 2 pi) = -RX(b)) changes nothing;
    two identical calls agree bit for bit."""
    n, p, edges = 30, 8, _bench_graph()
    a = I.uniform_params(2 * p, 3, 0.0, float(np.pi))
    g, b = a[:p], a[p:]
    q = Q.QAOA(n, edges, p, 0.5, Q.C64)
    psi, lam = Q.State(n, Q.C64), Q.State(n, Q.C64)
    sc = float(len(edges))
    # held to the energy's bound tol * |E| (tighter than the rule's bounds)
    te = tg = tb = TOL[0] * sc
    E0, dg0, db0 = q.expectation_with_grad(psi, lam, g, b)
    E1, dg1, db1 = q.expectation_with_grad(psi, lam, g, b)
    assert E0 == E1 and np.array_equal(dg0, dg1) and np.array_equal(db0, db1)
    assert abs(E0) <= sc
    Em, dgm, dbm = q.expectation_with_grad(psi, lam, -g, -b)
    check("qaoa30 p8 E(-theta)", abs(Em - E0), te)
    check("qaoa30 p8 dgamma(-theta)", np.abs(dgm + dg0), tg)
    check("qaoa30 p8 dbeta(-theta)", np.abs(dbm + db0), tb)
    b2 = b.copy()
    b2[3] += 2 * math.pi
    Es, dgs, dbs = q.expectation_with_grad(psi, lam, g, b2)
    check("qaoa30 p8 E(beta + 2 pi)", abs(Es - E0), te)
    check("qaoa30 p8 dgamma(beta + 2 pi)", np.abs(dgs - dg0), tg)
    check("qaoa30 p8 dbeta(beta + 2 pi)", np.abs(dbs - db0), tb)


def _inverse(circ):
    inv = []
    for gt in reversed(circ.gates):
        if gt.kind in ("RX", "RY", "RZ"):
            inv.append(I.Gate(gt.kind, gt.targets, gt.ctrls, gt.param, -gt.coef, -gt.const))
        else:  # H, X, Z (with or without controls) are their own inverses
            inv.append(gt)
    return I.Circuit(circ.n_qubits, inv, circ.n_params)


@pytest.mark.parametrize("dt,fuse", [(0, 0), (0, -1), (1, 0)])
def test_random28_then_inverse_returns_to_zero(Q, dt, fuse):
    """The 28-qubit, 500-gate random circuit (seed 2): the norm stays 1 and the
    circuit followed by its inverse returns |0...0> (fused passes and one kernel
    per gate, both precisions)."""
    n = 28
    circ = I.random_circuit(n, 500, 2)
    s = Q.State(n, dt).set_basis(0)
    c = Q.circuit_from(circ).finalize(dt, fuse=fuse)
    c.apply(s)
    # ||psi + d||^2 - 1 <= 2 ||d|| + ||d||^2 with ||d|| <= tol
    tag = f"random28 dt={dt} fuse={fuse}"
    check(tag + " norm", abs(s.norm2() - 1.0), 2 * TOL[dt] + TOL[dt] ** 2)
    ci = Q.circuit_from(_inverse(circ)).finalize(dt, fuse=fuse)
    ci.apply(s)
    amp = s.amplitudes
    a0 = complex(amp[0].item())
    # circuit and inverse: ||d|| <= 2 tol, so |a0 - 1| <= 2 tol and the rest of
    # the weight sum_{x != 0} |psi_x|^2 = ||d_rest||^2 <= (2 tol)^2
    check(tag + " inverse amplitude 0", abs(a0 - 1.0), 2 * TOL[dt])
    rest = float(s.norm2() - abs(a0) ** 2)
    check(tag + " inverse rest weight", max(rest, 0.0), (2 * TOL[dt]) ** 2 + 4 * np.finfo(np.float64).eps)


def test_batched_vqe_workload_sampled_instances(Q):
    """The 2048-instance batched workload (seed 4) in one persistent launch;
    six sampled instances (the largest qubit count among them) against the
    oracle's adjoint gradient."""
    inst = I.batched_vqe(2048, seed=4)
    b = Q.Batch(inst, Q.C64)
    e, g = b.expectation_with_grad([it.params for it in inst])
    nq = np.array([it.circuit.n_qubits for it in inst])
    depth = np.array([it.circuit.n_params // (2 * it.circuit.n_qubits) for it in inst])
    picks = [int(np.argmin(nq)), 7, 100, 1500]
    big = np.where(nq == nq.max())[0]
    picks.append(int(big[np.argmin(depth[big])]))
    picks.append(int(np.where(nq == 16)[0][0]))
    for i in picks:
        it = inst[i]
        psi0 = O.zero_state(it.circuit.n_qubits)
        E, G = O.adjoint_gradient(it.circuit, it.ham, it.params, psi0)
        check(f"batch2048 instance {i} energy", abs(e[i] - E), energy_tol(0, it.ham))
        check(f"batch2048 instance {i} grad", np.abs(g[i] - G), grad_tol(0, it.ham, it.circuit))


def _sweep_amplitude(n, x, rz, cnots, czs):
    """Amplitude at index x after H on every qubit of |0..0>, RZ(rz[q]) on every
    qubit, the CNOTs (c, t) in order, then CZ on each pair: CNOTs and CZs map a
    product state to a phased permutation of it, so the amplitude is written out
    from the definitions (RZ(a) = diag(e^{-ia/2}, e^{ia/2}))."""
    phase = 0.0
    for c, t in czs:
        if (x >> c) & 1 and (x >> t) & 1:
            phase += math.pi
    for c, t in reversed(cnots):  # undo the permutation back to the product state
        if (x >> c) & 1:
            x ^= 1 << t
    for q in range(n):
        phase += rz[q] / 2 if (x >> q) & 1 else -rz[q] / 2
    return 2.0 ** (-n / 2) * complex(math.cos(phase), math.sin(phase))


@pytest.mark.parametrize("dt,n", [(0, 30), (1, 29)])
def test_per_gate_sweep_at_full_size(Q, dt, n):
    """The single-gate kernels bench.py's gate sweep times, at its size: H, RZ,
    controlled X and controlled Z on every qubit (the paired, qubit-0, controlled
    and diagonal paths), checked on 4096 sampled amplitudes against the closed
    form and on the norm."""
    import torch
    rng = np.random.default_rng(7)
    rz = rng.uniform(-np.pi, np.pi, n)
    cnots = [(q, (q + 1) % n) for q in range(n)]
    czs = [((q + 2) % n, q) for q in range(n)]
    gates = [I.Gate("H", (q,)) for q in range(n)]
    gates += [I.Gate("RZ", (q,), const=float(rz[q])) for q in range(n)]
    gates += [I.Gate("X", (t,), (c,)) for c, t in cnots]
    gates += [I.Gate("Z", (t,), (c,)) for c, t in czs]
    c = Q.circuit_from(I.Circuit(n, gates)).finalize(dt, fuse=-1)
    s = Q.State(n, dt)
    s.set_basis(0)
    c.apply(s, [])
    idx = np.concatenate([np.arange(64), (1 << n) - 1 - np.arange(64), rng.integers(0, 1 << n, 3968)])
    got = s.amplitudes[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    want = np.array([_sweep_amplitude(n, int(x), rz, cnots, czs) for x in idx])
    # a sampled amplitude: its share tol * 2^(-n/2) of the 2-norm bound
    check(f"gate sweep n={n} dt={dt} sampled amplitudes", np.abs(got - want), TOL[dt] * 2.0 ** (-n / 2))
    check(f"gate sweep n={n} dt={dt} norm", abs(s.norm2() - 1.0), 2 * TOL[dt] + TOL[dt] ** 2)
    del s
    torch.cuda.empty_cache()
