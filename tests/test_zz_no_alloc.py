"""qs_expectation_noalloc: the allocation-free expectation entry point.

It is for callers whose device memory belongs to another allocator (or who
cannot afford the synchronisation of cudaMalloc/cudaFree), so the library must
not allocate on their behalf.  It must give the same energy as qs_expectation,
call after call, although every call reuses the same fixed working memory.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2406_17248_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {0: 5e-5, 1: 1e-11}


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
    scale = max(1.0, float(np.abs(ham.coef).sum()))
    s = Q.State(n, dt).set_qs(I.random_state(n, 290 + n))
    want = Q.expectation(s, Q.Hamiltonian(ham))
    want_other = Q.expectation(s, Q.Hamiltonian(other))
    first = Q.expectation_noalloc(s, ham)
    second = Q.expectation_noalloc(s, ham)
    assert abs(first - want) < TOL[dt] * scale
    assert abs(second - want) < TOL[dt] * scale
    # a different, smaller Hamiltonian right after: nothing stale from the last call leaks in
    got_other = Q.expectation_noalloc(s, other)
    assert abs(got_other - want_other) < TOL[dt] * max(1.0, float(np.abs(other.coef).sum()))


def test_noalloc_rejects_more_terms_than_its_fixed_memory(Q):
    n = 6
    ham = I.random_pauli_sum(n, 4097, seed=5)
    s = Q.State(n, 0).set_basis(0)
    with pytest.raises(Q.QSimError, match="at most 4096"):
        Q.expectation_noalloc(s, ham)
