"""GPU parity of dense k-qubit blocks (qs_apply_matrix) against the FP64 oracle:
the CUDA-core path in both precisions for k = 1..6, the tcgen05 tensor-core
path (complex64, k = 4, 5) on several target layouts and at the 28-qubit size
on sampled rows, and the argument checks."""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {0: 5e-5, 1: 1e-11}  # max-abs amplitude error: complex64, complex128


@pytest.fixture(scope="module")
def Q():
    from paper_2406_17248_gb300 import qsim
    qsim.lib()
    return qsim


def _unitary(k, seed):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    return np.linalg.qr(z)[0]


def _run(Q, n, dt, targets, U, engine, seed):
    psi0 = I.random_state(n, seed)
    s = Q.State(n, dt).set_qs(psi0)
    Q.apply_matrix(s, targets, U, engine)
    got = s.get_qs().astype(np.complex128)
    want = O.apply_gate(psi0.astype(np.complex64 if dt == Q.C64 else np.complex128).astype(np.complex128), n, U,
                        list(targets))
    return np.max(np.abs(got - want))


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_cuda_core_blocks(Q, dt, k):
    rng = np.random.default_rng(10 * k + dt)
    for n, seed in ((k, 1), (max(k, 4) + 1, 2), (11, 3)):
        if n < k:
            continue
        targets = [int(t) for t in rng.permutation(n)[:k]]
        assert _run(Q, n, dt, targets, _unitary(k, seed), 1, seed) <= TOL[dt]


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("layout", ["low", "high", "mixed", "spread"])
def test_tensor_core_blocks(Q, k, layout):
    n = {"low": k + 7, "high": 13, "mixed": 14, "spread": 16}[layout]
    rng = np.random.default_rng(k)
    targets = {"low": list(range(k)), "high": list(range(n - k, n))[::-1],
               "mixed": [0, 3, 9, 13, 7][:k], "spread": [int(t) for t in rng.permutation(n)[:k]]}[layout]
    err = _run(Q, n, Q.C64, targets, _unitary(k, 7 + k), 2, 5)
    assert err <= TOL[0]
    assert err <= 2e-6  # float32-level: the head/tail split keeps ~21 bits per product


@pytest.mark.parametrize("k", [4, 5])
def test_tensor_core_blocks_many_tiles_per_cta(Q, k):
    """21 qubits: 512 (k = 5) / 1024 (k = 4) tiles of 128 rows over one CTA per
    SM, so every CTA runs several tiles through its two operand stages and two
    tensor-memory accumulators (the pipeline's parity bookkeeping)."""
    n = 21
    targets = [1, 6, 11, 16, 20][:k]
    err = _run(Q, n, Q.C64, targets, _unitary(k, 17 + k), 2, 9)
    assert err <= 2e-6


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("pos", [1, 2, 4])
def test_tensor_core_blocks_qubit0_not_first(Q, k, pos):
    """Qubit 0 listed at another position than first: the library lists it
    first with the matrix's index bits permuted to match (so that column pairs
    move as 16-byte words); the result is the same operator on the same bits,
    for the many-tile launch and for the cuda-core engine."""
    if pos >= k:
        pytest.skip("position beyond k")
    n = 21
    targets = [1, 6, 11, 16, 20][:k]
    targets[pos] = 0
    U = _unitary(k, 40 + 3 * k + pos)
    assert _run(Q, n, Q.C64, targets, U, 2, 11) <= 2e-6
    assert _run(Q, 12, Q.C64, [t % 12 for t in targets], U, 1, 12) <= TOL[0]


def test_tensor_core_identity_and_permutation(Q):
    n, k = 13, 5
    psi0 = I.random_state(n, 9).astype(np.complex64)
    s = Q.State(n, Q.C64).set_qs(psi0)
    Q.apply_matrix(s, list(range(2, 7)), np.eye(1 << k), 2)
    assert np.max(np.abs(s.get_qs() - psi0)) <= 1e-6 * np.max(np.abs(psi0))
    perm = np.random.default_rng(1).permutation(1 << k)
    P = np.eye(1 << k)[perm]
    s.set_qs(psi0)
    Q.apply_matrix(s, [12, 0, 5, 8, 3], P, 2)
    want = O.apply_gate(psi0.astype(np.complex128), n, P, [12, 0, 5, 8, 3])
    assert np.max(np.abs(s.get_qs() - want)) <= 1e-6 * np.max(np.abs(psi0))


def test_tensor_core_full_size_sampled(Q):
    """28 qubits complex64 (2 GiB): the state comes from an index-addressable
    seeded generator; 96 sampled rows are checked against the oracle's block
    applied to the same rows."""
    n, k = 28, 5
    targets = [0, 4, 11, 19, 27]
    U = _unitary(k, 3)
    s = Q.State(n, Q.C64)
    amp = s.amplitudes
    chunk = 1 << 24
    for c0 in range(0, 1 << n, chunk):
        a = I.hashed_amplitudes(np.arange(c0, c0 + chunk, dtype=np.uint64), 11, n).astype(np.complex64)
        amp[c0:c0 + chunk].copy_(torch.from_numpy(a))
    Q.apply_matrix(s, targets, U, 2)
    others = [q for q in range(n) if q not in targets]
    rows = np.random.default_rng(4).integers(0, 1 << (n - k), size=96)
    tmask = [sum(((j >> b) & 1) << targets[b] for b in range(k)) for j in range(1 << k)]
    worst, scale = 0.0, 0.0
    for r in rows:
        base = sum(((int(r) >> b) & 1) << others[b] for b in range(n - k))
        idx = np.array([base | t for t in tmask], dtype=np.uint64)
        x = I.hashed_amplitudes(idx, 11, n).astype(np.complex64).astype(np.complex128)
        want = O.apply_gate(x, k, U, list(range(k)))
        got = amp[torch.as_tensor(idx.astype(np.int64), device="cuda")].cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - want))))
        scale = max(scale, float(np.max(np.abs(want))))
    # amplitudes of a 28-qubit state are ~1e-4: the bound is relative to the
    # largest sampled amplitude, at float32 level
    assert worst <= 2e-6 * scale


def test_argument_checks(Q):
    s = Q.State(10, Q.C64)
    s128 = Q.State(10, Q.C128)
    with pytest.raises(Q.QSimError):
        Q.apply_matrix(s128, [0, 1, 2, 3], np.eye(16), 2)  # tensor cores need complex64
    with pytest.raises(Q.QSimError):
        Q.apply_matrix(s, [0, 1, 2, 3, 4, 5, 6], np.eye(128), 1)  # k > 6
    with pytest.raises(Q.QSimError):
        Q.apply_matrix(s, [0, 1, 1, 3], np.eye(16), 1)  # repeated target
    with pytest.raises(Q.QSimError):
        Q.apply_matrix(s, [0, 1, 2, 10], np.eye(16), 1)  # out of range
    with pytest.raises(Q.QSimError):
        Q.apply_matrix(s, [0, 1, 2, 3, 4], np.eye(32), 2)  # needs n - k >= 7
