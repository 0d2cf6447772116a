"""Parity beyond the benchmark sizes, where every index of the state needs more
than 32 bits: the 32-qubit depth-1 QAOA energy and gradient against the closed
form, and a 33-qubit (68.7 GB) complex64 product state through the fused tile
passes and the per-gate kernels against its amplitudes written out in closed
form on sampled indices.  Skipped when the GPU has too little free memory."""
import math

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 5e-5  # complex64


@pytest.fixture(scope="module")
def Q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def _need_free(gb):
    import torch
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < gb * 1e9:
        pytest.skip(f"needs {gb} GB of free device memory")


def test_qaoa32_depth1_against_closed_form(Q):
    """32 qubits (psi, lam and the reverse sweep's second buffer: 3 x 34.4 GB):
    E and both gradient entries against the closed form and its central
    differences."""
    _need_free(120)
    n, edges = 32, I.random_regular_graph(32, 3, 7)
    q = Q.QAOA(n, edges, 1, 0.5, Q.C64)
    psi, lam = Q.State(n, Q.C64), Q.State(n, Q.C64)
    g, b = 0.83, -0.41
    E, dg, db = q.expectation_with_grad(psi, lam, [g], [b])
    f = lambda gg, bb: O.qaoa_p1_energy_closed_form(n, edges, gg, bb, 0.5)
    h = 1e-5
    sc = len(edges)
    assert abs(E - f(g, b)) <= TOL * sc
    assert abs(dg[0] - (f(g + h, b) - f(g - h, b)) / (2 * h)) <= TOL * sc
    assert abs(db[0] - (f(g, b + h) - f(g, b - h)) / (2 * h)) <= TOL * sc
    del psi, lam, q


def _product_amplitudes(theta, idx):
    """RY(theta_q) on every qubit of |0..0>: amplitude of x is the product over q
    of cos(theta_q / 2) (bit q of x clear) or sin(theta_q / 2) (set)."""
    a = np.ones(idx.size)
    for q, t in enumerate(theta):
        bit = (idx >> np.uint64(q)) & np.uint64(1)
        a *= np.where(bit == 1, math.sin(t / 2), math.cos(t / 2))
    return a


def test_33_qubit_state_fused_and_per_gate(Q):
    import torch
    _need_free(80)
    n = 33
    rng = np.random.default_rng(33)
    theta = rng.uniform(-math.pi, math.pi, n)
    idx = np.concatenate([rng.integers(0, 1 << n, size=120, dtype=np.uint64),
                          np.array([0, (1 << n) - 1, 1 << 32, (1 << 32) - 1, (1 << 31) + 5], dtype=np.uint64)])
    s = Q.State(n, Q.C64)
    s.set_basis(0)
    circ = I.Circuit(n, [I.Gate("RY", (q,), const=float(theta[q])) for q in range(n)])
    Q.circuit_from(circ).finalize(Q.C64).apply(s)
    amp = s.amplitudes
    tix = torch.as_tensor(idx.astype(np.int64), device="cuda")
    want = _product_amplitudes(theta, idx)
    scale = float(np.abs(want).max())
    got = amp[tix].cpu().numpy().astype(np.complex128)
    assert np.abs(got - want).max() <= 1e-5 * scale
    assert abs(s.norm2() - 1.0) < TOL
    # per-gate kernels: CNOT (control 32, target 0), then RZ(phi) on qubit 32
    phi = 0.7
    per = I.Circuit(n, [I.Gate("X", (0,), (32,)), I.Gate("RZ", (32,), const=phi)])
    Q.circuit_from(per).finalize(Q.C64, fuse=-1).apply(s)
    hi = (idx >> np.uint64(32)) & np.uint64(1)
    src = np.where(hi == 1, idx ^ np.uint64(1), idx)
    want2 = _product_amplitudes(theta, src) * np.where(hi == 1, np.exp(0.5j * phi), np.exp(-0.5j * phi))
    got2 = amp[tix].cpu().numpy().astype(np.complex128)
    assert np.abs(got2 - want2).max() <= 1e-5 * scale
    del s, amp
    torch.cuda.empty_cache()
