"""FP64 CPU oracle for the state-vector VQA hot path (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm may import this module.  The product (the CUDA library and its
Python binding) never calls it and shares no code with it.

It is a plain, slow, obviously-correct restatement of what the paper defines,
in numpy complex128:

* state: 2^n amplitudes, little endian -- qubit q is bit q of the index
  (§2.6, "Basic Usage of Simulator").
* gate matrices: X, Y, Z, H (§2.3.2), RX, RY, RZ = exp(-i theta P / 2) (§2.3.3);
  S, T, PhaseShift, SWAP, RXX, RYY, RZZ are the textbook definitions (the paper
  uses but does not print them; RZZ(theta) = exp(-i theta/2 Z(x)Z), the same
  half-angle convention as RX/RY/RZ).
* controls (§2.3.5): U acts on the targets where every control bit is 1.
* Pauli strings and Hamiltonians (§2.5.1), apply_hamiltonian (§2.6.1),
  expectation <psi|H|psi> (§2.6.2).
* gradient: the adjoint method (named in §7.2; the same forward/backward
  structure is written out for GRAPE in §6.4), parameter shift and central
  finite differences as independent checks (§4.1).
* sampling (§2.6.3): inverse-CDF draws with uniforms from splitmix64
  (Steele, Lea & Flood 2014, the published constants).
* QuPack QAOA (§6.2): |+>^n, per layer exp(-i gamma_l sum ZZ) then RX(beta_l).

Two independent appliers exist: ``apply_gate`` (tensor-axis contraction of the
pairwise definition, any n) and ``dense_unitary`` (explicit 2^n x 2^n Kronecker
products, n <= 10).  Tests pin them against each other and against values the
paper prints.

Parity: every function here is pinned by a ``-m "not gpu"`` test in
tests/test_oracle_pins.py or tests/test_oracle_properties.py -- values the
paper prints, closed forms, brute force or an independent algorithm.
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

import numpy as np

from paper_2406_17248_gb300.inputs import Circuit, Gate, PauliSum

C128 = np.complex128

# --------------------------------------------------------------------------- gate matrices

_I2 = np.eye(2, dtype=C128)
_X = np.array([[0, 1], [1, 0]], dtype=C128)          # §2.3.2
_Y = np.array([[0, -1j], [1j, 0]], dtype=C128)       # §2.3.2
_Z = np.array([[1, 0], [0, -1]], dtype=C128)         # §2.3.2
_H = np.array([[1, 1], [1, -1]], dtype=C128) / math.sqrt(2.0)  # §2.3.2


def _kron_targets(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Matrix of a on targets[0] and b on targets[1]; basis index = bit0 + 2*bit1."""
    return np.kron(b, a)


def gate_matrix(kind: str, theta: float = 0.0, matrix=None) -> np.ndarray:
    """Unitary of one gate on its targets (basis index sum_j bit(targets[j]) << j)."""
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    if kind == "I":
        return _I2.copy()
    if kind == "X":
        return _X.copy()
    if kind == "Y":
        return _Y.copy()
    if kind == "Z":
        return _Z.copy()
    if kind == "H":
        return _H.copy()
    if kind == "S":
        return np.diag([1, 1j]).astype(C128)
    if kind == "SDG":
        return np.diag([1, -1j]).astype(C128)
    if kind == "T":
        return np.diag([1, np.exp(1j * math.pi / 4)]).astype(C128)
    if kind == "TDG":
        return np.diag([1, np.exp(-1j * math.pi / 4)]).astype(C128)
    if kind == "SWAP":
        m = np.zeros((4, 4), dtype=C128)
        m[0, 0] = m[3, 3] = 1
        m[1, 2] = m[2, 1] = 1
        return m
    # §2.3.3: R_P(theta) = cos(theta/2) I - i sin(theta/2) P
    if kind == "RX":
        return c * _I2 - 1j * s * _X
    if kind == "RY":
        return c * _I2 - 1j * s * _Y
    if kind == "RZ":
        return c * _I2 - 1j * s * _Z
    if kind == "PS":
        return np.diag([1, np.exp(1j * theta)]).astype(C128)
    if kind == "RXX":
        return c * np.eye(4, dtype=C128) - 1j * s * _kron_targets(_X, _X)
    if kind == "RYY":
        return c * np.eye(4, dtype=C128) - 1j * s * _kron_targets(_Y, _Y)
    if kind == "RZZ":
        return c * np.eye(4, dtype=C128) - 1j * s * _kron_targets(_Z, _Z)
    if kind == "MATRIX":
        m = np.asarray(matrix, dtype=C128)
        d = int(round(math.sqrt(m.size)))
        return m.reshape(d, d)
    raise ValueError(f"unknown gate kind {kind!r}")


def gate_matrix_derivative(kind: str, theta: float) -> np.ndarray:
    """d U(theta) / d theta, written from the definitions above."""
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    dc, ds = -0.5 * s, 0.5 * c
    if kind == "RX":
        return dc * _I2 - 1j * ds * _X
    if kind == "RY":
        return dc * _I2 - 1j * ds * _Y
    if kind == "RZ":
        return dc * _I2 - 1j * ds * _Z
    if kind == "PS":
        return np.diag([0, 1j * np.exp(1j * theta)]).astype(C128)
    if kind == "RXX":
        return dc * np.eye(4, dtype=C128) - 1j * ds * _kron_targets(_X, _X)
    if kind == "RYY":
        return dc * np.eye(4, dtype=C128) - 1j * ds * _kron_targets(_Y, _Y)
    if kind == "RZZ":
        return dc * np.eye(4, dtype=C128) - 1j * ds * _kron_targets(_Z, _Z)
    raise ValueError(f"gate kind {kind!r} has no parameter")


def gate_unitary(g: Gate, params: Sequence[float]) -> np.ndarray:
    return gate_matrix(g.kind, g.angle(params), g.matrix)


# --------------------------------------------------------------------------- states

def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=C128)
    psi[0] = 1.0
    return psi


def basis_state(n: int, index: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=C128)
    psi[index] = 1.0
    return psi


def plus_state(n: int) -> np.ndarray:
    return np.full(1 << n, 2.0 ** (-n / 2), dtype=C128)


# --------------------------------------------------------------------------- applier 1: axes

def _apply_on_subspace(psi: np.ndarray, n: int, U: np.ndarray, targets: Sequence[int],
                       ctrls: Sequence[int], out: np.ndarray) -> None:
    """out[control-satisfied block] = U (x) I acting on psi's block (pairwise rule).

    The state is viewed as an n-axis tensor whose axis a holds qubit n-1-a (the
    little-endian index read most-significant first)."""
    k = len(targets)
    src = psi.reshape((2,) * n)
    dst = out.reshape((2,) * n)
    sl = [slice(None)] * n
    for cq in ctrls:
        sl[n - 1 - cq] = 1
    sub_src = src[tuple(sl)]
    sub_dst = dst[tuple(sl)]
    rest = [q for q in range(n - 1, -1, -1) if q not in ctrls]  # qubit of each remaining axis
    pos = [rest.index(t) for t in targets]
    # U reshaped to (2,)*2k: axes (out bit k-1 .. out bit 0, in bit k-1 .. in bit 0)
    Ut = U.reshape((2,) * (2 * k))
    in_axes = list(range(2 * k - 1, k - 1, -1))  # in bit 0, in bit 1, ...
    res = np.tensordot(Ut, sub_src, axes=(in_axes, pos))
    # res axes: out bit k-1, ..., out bit 0, remaining axes of sub_src without pos
    res = np.moveaxis(res, list(range(k)), [pos[j] for j in range(k - 1, -1, -1)])
    sub_dst[...] = res


def apply_gate(psi: np.ndarray, n: int, U: np.ndarray, targets: Sequence[int],
               ctrls: Sequence[int] = ()) -> np.ndarray:
    """psi <- (controlled) U on targets; returns a new array."""
    out = psi.copy()
    _apply_on_subspace(psi, n, U, targets, ctrls, out)
    return out


def apply_on_control_subspace_only(psi: np.ndarray, n: int, M: np.ndarray,
                                   targets: Sequence[int], ctrls: Sequence[int]) -> np.ndarray:
    """(P_ctrl (x) M) psi: M on the control-satisfied block, zero elsewhere."""
    out = np.zeros_like(psi)
    _apply_on_subspace(psi, n, M, targets, ctrls, out)
    return out


def evolve(circ: Circuit, params: Sequence[float], psi0: np.ndarray) -> np.ndarray:
    psi = psi0.astype(C128, copy=True)
    for g in circ.gates:
        psi = apply_gate(psi, circ.n_qubits, gate_unitary(g, params), g.targets, g.ctrls)
    return psi


# --------------------------------------------------------------------------- applier 2: dense

def _embed(n: int, U: np.ndarray, targets: Sequence[int]) -> np.ndarray:
    """2^n x 2^n matrix of U on `targets` (identity elsewhere), by explicit sums of
    Kronecker products of single-qubit operators |a><b| (qubit 0 right-most)."""
    k = len(targets)
    full = np.zeros((1 << n, 1 << n), dtype=C128)
    for row in range(1 << k):
        for col in range(1 << k):
            if U[row, col] == 0:
                continue
            factors = []
            for q in range(n - 1, -1, -1):
                if q in targets:
                    j = list(targets).index(q)
                    a, b = (row >> j) & 1, (col >> j) & 1
                    e = np.zeros((2, 2), dtype=C128)
                    e[a, b] = 1
                    factors.append(e)
                else:
                    factors.append(_I2)
            term = factors[0]
            for f in factors[1:]:
                term = np.kron(term, f)
            full += U[row, col] * term
    return full


def dense_gate_unitary(n: int, U: np.ndarray, targets: Sequence[int], ctrls: Sequence[int] = ()) -> np.ndarray:
    """U_full = (I - P) + P (U on targets), P = projector onto all controls = 1."""
    if n > 10:
        raise ValueError("dense applier is for n <= 10")
    Ufull = _embed(n, U, targets)
    if not ctrls:
        return Ufull
    P = np.eye(1, dtype=C128)
    for q in range(n - 1, -1, -1):
        P = np.kron(P, np.diag([0, 1]).astype(C128) if q in ctrls else _I2)
    I = np.eye(1 << n, dtype=C128)
    return (I - P) + P @ Ufull


def dense_circuit_unitary(circ: Circuit, params: Sequence[float]) -> np.ndarray:
    n = circ.n_qubits
    W = np.eye(1 << n, dtype=C128)
    for g in circ.gates:
        W = dense_gate_unitary(n, gate_unitary(g, params), g.targets, g.ctrls) @ W
    return W


# --------------------------------------------------------------------------- Pauli sums

def pauli_string_matrix(n: int, xmask: int, zmask: int) -> np.ndarray:
    """Dense matrix of one Pauli string (§2.5.1), qubit 0 right-most factor."""
    m = np.eye(1, dtype=C128)
    for q in range(n - 1, -1, -1):
        x, z = (xmask >> q) & 1, (zmask >> q) & 1
        p = _I2 if not (x or z) else (_X if x and not z else (_Z if z and not x else _Y))
        m = np.kron(m, p)
    return m


def hamiltonian_matrix(ham: PauliSum) -> np.ndarray:
    d = 1 << ham.n_qubits
    Hm = np.zeros((d, d), dtype=C128)
    for x, z, c in zip(ham.xmask, ham.zmask, ham.coef):
        Hm += c * pauli_string_matrix(ham.n_qubits, int(x), int(z))
    return Hm


def _popcount_parity(v: np.ndarray) -> np.ndarray:
    v = v.copy()
    par = np.zeros(v.shape, dtype=np.int64)
    while np.any(v):
        par ^= (v & 1).astype(np.int64)
        v >>= np.uint64(1)
    return par


def apply_pauli_string(psi: np.ndarray, n: int, xmask: int, zmask: int) -> np.ndarray:
    """P|x> = i^{#Y} (-1)^{popcount(x & zmask)} |x XOR xmask>  (Y = i X Z)."""
    idx = np.arange(1 << n, dtype=np.uint64)
    ny = bin(xmask & zmask).count("1")
    sign = 1 - 2 * _popcount_parity(idx & np.uint64(zmask))
    out = np.zeros_like(psi)
    out[(idx ^ np.uint64(xmask)).astype(np.int64)] = (1j ** ny) * sign * psi
    return out


def apply_hamiltonian(psi: np.ndarray, ham: PauliSum) -> np.ndarray:
    """H psi, unnormalised (§2.6.1 apply_hamiltonian)."""
    out = np.zeros_like(psi)
    for x, z, c in zip(ham.xmask, ham.zmask, ham.coef):
        out += c * apply_pauli_string(psi, ham.n_qubits, int(x), int(z))
    return out


def expectation(psi: np.ndarray, ham: PauliSum) -> float:
    """<psi|H|psi> for Hermitian H (real coefficients): the real part (§2.6.2)."""
    return float(np.real(np.vdot(psi, apply_hamiltonian(psi, ham))))


def inner_product(bra: np.ndarray, ket: np.ndarray) -> complex:
    return complex(np.vdot(bra, ket))


# --------------------------------------------------------------------------- gradients

def expectation_of_circuit(circ: Circuit, ham: PauliSum, params, psi0) -> float:
    return expectation(evolve(circ, params, psi0), ham)


def adjoint_gradient(circ: Circuit, ham: PauliSum, params: Sequence[float], psi0: np.ndarray):
    """Energy and dE/dparams by the adjoint method.

    psi = U_N..U_1 psi0, E = <psi|H|psi>, lam = H psi.  For k = N..1:
    psi <- U_k^dag psi (now the state before gate k);
    if gate k depends on parameter p with d angle/dp = coef:
        grad[p] += coef * 2 Re <lam| (P_ctrl (x) dU_k/dtheta) |psi>;
    lam <- U_k^dag lam.
    """
    n = circ.n_qubits
    psi = evolve(circ, params, psi0)
    E = expectation(psi, ham)
    lam = apply_hamiltonian(psi, ham)
    grad = np.zeros(circ.n_params, dtype=np.float64)
    for g in reversed(circ.gates):
        U = gate_unitary(g, params)
        Ud = U.conj().T
        psi = apply_gate(psi, n, Ud, g.targets, g.ctrls)
        if g.param >= 0:
            dU = gate_matrix_derivative(g.kind, g.angle(params))
            dpsi = apply_on_control_subspace_only(psi, n, dU, g.targets, g.ctrls)
            grad[g.param] += g.coef * 2.0 * np.real(np.vdot(lam, dpsi))
        lam = apply_gate(lam, n, Ud, g.targets, g.ctrls)
    return E, grad


def _with_angle(g: Gate, new_angle: float) -> Gate:
    return Gate(g.kind, g.targets, g.ctrls, -1, 1.0, new_angle, g.matrix)


def parameter_shift_gradient(circ: Circuit, ham: PauliSum, params, psi0):
    """Two-term shift rule per gate occurrence, exact for generators with two
    eigenvalues +-1/2 (uncontrolled RX/RY/RZ/RXX/RYY/RZZ and PS); chained by coef."""
    grad = np.zeros(circ.n_params, dtype=np.float64)
    for k, g in enumerate(circ.gates):
        if g.param < 0:
            continue
        if g.ctrls:
            raise ValueError("two-term shift rule does not hold for controlled rotations")
        a = g.angle(params)
        vals = []
        for shift in (+math.pi / 2, -math.pi / 2):
            gates = list(circ.gates)
            gates[k] = _with_angle(g, a + shift)
            vals.append(expectation_of_circuit(Circuit(circ.n_qubits, gates, circ.n_params), ham, params, psi0))
        grad[g.param] += g.coef * 0.5 * (vals[0] - vals[1])
    return grad


def finite_difference_gradient(circ: Circuit, ham: PauliSum, params, psi0, h: float = 1e-6):
    params = np.asarray(params, dtype=np.float64)
    grad = np.zeros(circ.n_params, dtype=np.float64)
    for p in range(circ.n_params):
        e = np.zeros_like(params)
        e[p] = h
        grad[p] = (expectation_of_circuit(circ, ham, params + e, psi0)
                   - expectation_of_circuit(circ, ham, params - e, psi0)) / (2 * h)
    return grad


# --------------------------------------------------------------------------- QAOA (§5.2, §6.2)

def cut_values(n: int, edges: Sequence[Tuple[int, int]]) -> np.ndarray:
    """C(x) = sum_{(i,j) in E} z_i z_j with z = 1 - 2 * bit (an integer per basis state)."""
    idx = np.arange(1 << n, dtype=np.int64)
    C = np.zeros(1 << n, dtype=np.int64)
    for a, b in edges:
        C += 1 - 2 * (((idx >> a) ^ (idx >> b)) & 1)
    return C


def qaoa_layers_state(n: int, edges, gamma, beta, gamma_scale: float = 1.0):
    """|+>^n, then per layer exp(-i gamma_scale*gamma_l * C) then RX(beta_l) on every qubit.
    gamma_scale = 1 is the QuPack form (§6.2); 0.5 is RZZ(gamma) per edge."""
    C = cut_values(n, edges).astype(np.float64)
    psi = plus_state(n)
    for g, b in zip(gamma, beta):
        psi = np.exp(-1j * gamma_scale * g * C) * psi
        rx = gate_matrix("RX", b)
        for q in range(n):
            psi = apply_gate(psi, n, rx, (q,))
    return psi


def qaoa_expectation_with_grad(n: int, edges, gamma, beta, gamma_scale: float = 1.0):
    """Energy <C> and its gradient w.r.t. every gamma_l and beta_l, by the adjoint
    method on the layer form (cost layer: generator gamma_scale*C, mixer layer:
    generator sum_q X_q / 2 with all qubits sharing beta_l)."""
    C = cut_values(n, edges).astype(np.float64)
    p = len(gamma)
    psi = qaoa_layers_state(n, edges, gamma, beta, gamma_scale)
    E = float(np.real(np.vdot(psi, C * psi)))
    lam = C * psi
    dg = np.zeros(p)
    db = np.zeros(p)
    for l in range(p - 1, -1, -1):
        rxd = gate_matrix("RX", beta[l]).conj().T
        # dE/dbeta_l = sum_q Im <lam| X_q |psi> (RX_q commutes with X_q, so every
        # term may be taken at the state after the whole mixer layer).
        for q in range(n):
            xpsi = apply_gate(psi, n, _X, (q,))
            db[l] += float(np.imag(np.vdot(lam, xpsi)))
        for q in range(n):
            psi = apply_gate(psi, n, rxd, (q,))
            lam = apply_gate(lam, n, rxd, (q,))
        # dE/dgamma_l = 2 Re <lam| (-i gamma_scale C) |psi> = 2 gamma_scale Im <lam|C|psi>
        dg[l] = 2.0 * gamma_scale * float(np.imag(np.vdot(lam, C * psi)))
        ph = np.exp(1j * gamma_scale * gamma[l] * C)
        psi = ph * psi
        lam = ph * lam
    return E, dg, db


def maxcut_brute_force(n: int, edges) -> int:
    C = cut_values(n, edges)
    return int((len(edges) - C.min()) // 2)


# --------------------------------------------------------------------------- sampling (§2.6.3)

_M64 = (1 << 64) - 1


def splitmix64(state: int) -> Tuple[int, int]:
    """One step of splitmix64: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def shot_uniform(seed: int, shot: int) -> float:
    """u_s in [0, 1): splitmix64 output for counter state seed + s*golden, top 53 bits."""
    state = (seed + shot * 0x9E3779B97F4A7C15) & _M64
    _, z = splitmix64(state)
    return (z >> 11) * (1.0 / (1 << 53))


def sample(psi: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Outcome s = smallest x with cdf(x) > u_s * cdf(last), cdf = prefix sums of |psi_x|^2."""
    p = np.abs(psi) ** 2
    cdf = np.cumsum(p)
    total = cdf[-1]
    u = np.array([shot_uniform(seed, s) for s in range(shots)], dtype=np.float64)
    return np.searchsorted(cdf, u * total, side="right").astype(np.uint64)


def qaoa_p1_energy_closed_form(n: int, edges, gamma: float, beta: float, gamma_scale: float = 1.0) -> float:
    """<sum_E Z_u Z_v> of depth-1 MaxCut QAOA in closed form (Wang, Hadfield,
    Jiang & Rieffel 2018, Theorem 1), valid for any n: for the state
    exp(-i b B) exp(-i g C)|+>^n with C = sum (1 - Z_u Z_v)/2 and B = sum X,
      <C_uv> = 1/2 + sin(4b) sin(g) (cos^du g + cos^dv g)/4
                   - sin^2(2b) cos^(du + dv - 2f) g (1 - cos^f 2g)/4,
    du = deg(u) - 1, dv = deg(v) - 1, f = triangles on the edge.  This
    module's layer exp(-i gamma_scale gamma sum ZZ) then RX(beta) is that state
    with g = -2 gamma_scale gamma and b = beta / 2 (global phases aside)."""
    g = -2.0 * gamma_scale * gamma
    b = beta / 2.0
    nb = [set() for _ in range(n)]
    for a, c in edges:
        nb[a].add(c)
        nb[c].add(a)
    total = 0.0
    for u, v in edges:
        du, dv, f = len(nb[u]) - 1, len(nb[v]) - 1, len(nb[u] & nb[v])
        cuv = (0.5 + 0.25 * math.sin(4 * b) * math.sin(g) * (math.cos(g) ** du + math.cos(g) ** dv)
               - 0.25 * math.sin(2 * b) ** 2 * math.cos(g) ** (du + dv - 2 * f) * (1 - math.cos(2 * g) ** f))
        total += 1.0 - 2.0 * cuv
    return total


def measure(psi: np.ndarray, n: int, qubit: int, seed: int):
    """Projective measurement of one qubit (the measurement gate of §2.3, with the
    outcome drawn as in sampling, §2.6.3): P1 = sum of |psi_x|^2 over x with the
    bit set, u = shot_uniform(seed, 0); outcome 0 iff P0 > u * total; the state is
    projected onto the outcome and renormalised.  Returns (outcome, new state, P1 / total)."""
    x = np.arange(psi.size, dtype=np.int64)
    prob = np.abs(psi) ** 2
    on = ((x >> qubit) & 1) == 1
    tot = float(prob.sum())
    p1 = float(prob[on].sum())
    p0 = tot - p1
    u = shot_uniform(seed, 0)
    outcome = 0 if p0 > u * tot else 1
    keep = on if outcome == 1 else ~on
    out = np.where(keep, psi, 0.0).astype(psi.dtype)
    pk = p1 if outcome == 1 else p0
    return outcome, out / math.sqrt(pk), p1 / tot


# --------------------------------------------------------------------------- DC-QAOA (§5.4)

def dcqaoa_state_by_definition(n: int, ham_prob: PauliSum, params: Sequence[float], p: int,
                               cd: bool = True) -> np.ndarray:
    """DC-QAOA state written from its definition in §5.4: start from H^n|0> (the
    ground state of -sum X, prepared by a Hadamard on every qubit), then per layer
    apply U_p(gamma) = exp(-i gamma H_prob), U_m(beta) = exp(-i beta sum_q X_q) and,
    with ``cd``, U_cd(alpha) = exp(-i alpha sum_q Y_q), each as the matrix
    exponential of the dense operator (scipy.linalg.expm; n <= 10).  Parameters
    per layer: (gamma, beta, alpha), or (gamma, beta) without ``cd``.  This is
    independent of any gate decomposition of the three evolutions."""
    from scipy.linalg import expm
    from paper_2406_17248_gb300.inputs import pauli_sum_from_strings
    if n > 10:
        raise ValueError("dense matrix exponentials are limited to n <= 10")
    Hp = hamiltonian_matrix(ham_prob)
    Hm = hamiltonian_matrix(pauli_sum_from_strings(n, [(1.0, f"X{q}") for q in range(n)]))
    Hcd = hamiltonian_matrix(pauli_sum_from_strings(n, [(1.0, f"Y{q}") for q in range(n)]))
    per = 3 if cd else 2
    psi = plus_state(n)
    for l in range(p):
        psi = expm(-1j * params[per * l] * Hp) @ psi
        psi = expm(-1j * params[per * l + 1] * Hm) @ psi
        if cd:
            psi = expm(-1j * params[per * l + 2] * Hcd) @ psi
    return psi


def dcqaoa_p1_energy_at_gamma0(n: int, J: float, h: float, alpha: float) -> float:
    """<H_prob> of one DC-QAOA layer with gamma = 0 and k = 0, in closed form.
    With gamma = 0 the state is a product: each qubit is exp(-i alpha Y)
    exp(-i beta X)|+>; the X evolution only multiplies |+> by a phase, and the Y
    evolution turns the Bloch vector (1, 0, 0) about the y axis by 2 alpha to
    (cos 2a, 0, -sin 2a).  So <Z_q> = -sin 2a, <Z_i Z_{i+1}> = sin^2 2a and
    E = -J (n - 1) sin^2(2a) + h n sin(2a), for every beta; at alpha = -pi/4 this is
    the ground energy -(J (n - 1) + h n) of the chain (J, h >= 0)."""
    s = math.sin(2.0 * alpha)
    return -J * (n - 1) * s * s + h * n * s


def ising_chain_min_energy_brute_force(n: int, J: float, h: float) -> float:
    """min over spin configurations z in {+1, -1}^n of -J sum z_i z_{i+1} - h sum z_i
    by enumeration (the diagonal of H_prob for k = 0, §5.4)."""
    best = math.inf
    for x in range(1 << n):
        z = [1 - 2 * ((x >> q) & 1) for q in range(n)]
        e = -J * sum(z[i] * z[i + 1] for i in range(n - 1)) - h * sum(z)
        best = min(best, e)
    return best


# --------------------------------------------------------------------------- generalised expectation (§2.6.2, §4.1)

def general_expectation(circ_r: Circuit, circ_l: Circuit, ham: PauliSum, params, psi0, phi0) -> complex:
    """E = <phi|U_l^dag H U_r|psi> (the generalised observable of §2.6.2 and §4.1):
    U_r applied to psi0, U_l to phi0, both with the same parameter vector."""
    r = evolve(circ_r, params, psi0)
    l = evolve(circ_l, params, phi0)
    return inner_product(l, apply_hamiltonian(r, ham))


def _derivative_states(circ: Circuit, params, psi0):
    """For every parametric gate k: (param, coef, U_N..U_{k+1} (P_ctrl (x) dU_k) U_{k-1}..U_1 psi0)."""
    n = circ.n_qubits
    out = []
    for k, g in enumerate(circ.gates):
        if g.param < 0:
            continue
        psi = psi0.astype(C128, copy=True)
        for j, h in enumerate(circ.gates):
            if j == k:
                dU = gate_matrix_derivative(h.kind, h.angle(params))
                psi = apply_on_control_subspace_only(psi, n, dU, h.targets, h.ctrls)
            else:
                psi = apply_gate(psi, n, gate_unitary(h, params), h.targets, h.ctrls)
        out.append((g.param, g.coef, psi))
    return out


def general_expectation_grad(circ_r: Circuit, circ_l: Circuit, ham: PauliSum, params, psi0, phi0):
    """E and dE/dparams (complex) by the product rule, one derivative circuit per
    parametric gate occurrence (no adjoint sweep):
      dE/dp = sum_{k in U_r, param p} coef_k <phi_l| H |d_k psi>
            + sum_{k in U_l, param p} coef_k <d_k phi| H |psi_r>,
    with d_k the circuit whose gate k is replaced by its derivative."""
    n_params = max(circ_r.n_params, circ_l.n_params)
    r = evolve(circ_r, params, psi0)
    l = evolve(circ_l, params, phi0)
    Hl = apply_hamiltonian(l, ham)
    Hr = apply_hamiltonian(r, ham)
    grad = np.zeros(n_params, dtype=C128)
    for p, coef, d in _derivative_states(circ_r, params, psi0):
        grad[p] += coef * np.vdot(Hl, d)
    for p, coef, d in _derivative_states(circ_l, params, phi0):
        grad[p] += coef * np.vdot(d, Hr)
    return inner_product(l, Hr), grad
