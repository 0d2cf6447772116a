"""qs_expectation_noalloc: the allocation-free expectation entry point.

It is for callers whose device memory belongs to another allocator (or who
cannot afford the synchronisation of cudaMalloc/cudaFree), so the library must
not allocate on their behalf.  It must give the same energy as qs_expectation,
call after call, although every call reuses the same fixed working memory; the
energy must match the FP64 oracle too (the two entry points share the Pauli-sum
kernel, so a fault in that kernel would pass the first comparison), and the
device's free memory must not move across repeated calls.
This file is collected last on purpose."""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I
from tolerance import check, energy_tol

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


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n", [3, 12, 20])
def test_noalloc_matches_expectation_on_two_calls_in_a_row(Q, dt, n):
    ham = I.random_pauli_sum(n, 40, seed=90 + n)
    other = I.random_pauli_sum(n, 7, seed=190 + n)
    psi0 = I.random_state(n, 290 + n)
    s = Q.State(n, dt).set_qs(psi0)
    want = Q.expectation(s, Q.Hamiltonian(ham))
    want_other = Q.expectation(s, Q.Hamiltonian(other))
    first = Q.expectation_noalloc(s, ham)
    second = Q.expectation_noalloc(s, ham)
    tag = f"noalloc n={n} dt={dt}"
    check(tag + " first", abs(first - want), energy_tol(dt, ham))
    check(tag + " second", abs(second - want), energy_tol(dt, ham))
    # a different, smaller Hamiltonian right after: nothing stale from the last call leaks in
    got_other = Q.expectation_noalloc(s, other)
    check(tag + " other", abs(got_other - want_other), energy_tol(dt, other))
    if n <= 12:  # the FP64 oracle on the state as stored (complex64 rounding included)
        stored = s.get_qs().astype(np.complex128)
        check(tag + " vs oracle", abs(first - O.expectation(stored, ham)), energy_tol(dt, ham))


def test_noalloc_leaves_free_device_memory_unchanged(Q):
    import torch
    n = 16
    ham = I.random_pauli_sum(n, 64, seed=3)
    s = Q.State(n, 0).set_qs(I.random_state(n, 4))
    Q.expectation_noalloc(s, ham)  # first call on the device: takes the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        Q.expectation_noalloc(s, ham)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_more_terms_than_its_fixed_memory(Q):
    n = 6
    ham = I.random_pauli_sum(n, 4097, seed=5)
    s = Q.State(n, 0).set_basis(0)
    with pytest.raises(Q.QSimError, match="at most 4096"):
        Q.expectation_noalloc(s, ham)
