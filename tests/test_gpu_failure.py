"""Failure detection without faulting the GPU: a bounded device-side wait on a
barrier that nothing releases gives up, reports QS_ERR_TIMEOUT through the C
ABI, and the context stays usable (a computation afterwards still matches the
oracle); host-made errors come back as status codes."""
import ctypes as C

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

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


def test_bounded_wait_times_out_and_context_survives(Q):
    flag = C.c_int(-1)
    st = Q.lib().qs_selftest_wait_timeout(C.byref(flag))
    assert st == 4 and flag.value == 1  # QS_ERR_TIMEOUT
    assert b"self-test" in Q.lib().qs_last_error()
    n = 10
    circ = I.random_mixed_circuit(n, 40, 8)
    x = I.uniform_params(circ.n_params, 1)
    s = Q.State(n, 1).set_basis(0)
    Q.circuit_from(circ).finalize(1).apply(s, x)
    assert np.abs(s.get_qs() - O.evolve(circ, x, O.zero_state(n))).max() < 1e-11


def test_host_made_errors_return_status(Q):
    s = Q.State(4, 0)
    with pytest.raises(Q.QSimError):
        Q.circuit_from(I.Circuit(5, [I.Gate("H", (0,))])).finalize(0).apply(s)  # qubit counts differ
    with pytest.raises(Q.QSimError, match="tile_bits"):
        Q.Circuit(4).add("H", [0]).finalize(0, tile_bits=3)
    # the state is still usable
    s.set_basis(3)
    assert abs(s.norm2() - 1.0) < 1e-6


def test_repeatable_bits_as_a_race_smoke_test(Q):
    """Every reduction has a fixed order, so two identical calls agree bit for
    bit (a data race would show up as run-to-run differences)."""
    n = 16
    circ = I.random_mixed_circuit(n, 80, 2)
    ham = I.random_pauli_sum(n, 10, 4)
    x = I.uniform_params(circ.n_params, 3)
    c = Q.circuit_from(circ).finalize(0, tile_bits=9)
    h = Q.Hamiltonian(ham)
    out = []
    for _ in range(2):
        psi, lam = Q.State(n, 0).set_basis(0), Q.State(n, 0)
        out.append(Q.expectation_with_grad(psi, lam, c, h, x))
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])
    eng = Q.trajectories_from(I.hea_circuit(8, 2), {0: [("depolarizing", (0.2,), 0)], 5: [("amplitude_damping", (0.3,), 2)]})
    e1 = eng.run(Q.Hamiltonian(I.chain_zz_x(8)), I.uniform_params(32, 1), 512, seed=4)
    e2 = eng.run(Q.Hamiltonian(I.chain_zz_x(8)), I.uniform_params(32, 1), 512, seed=4)
    assert np.array_equal(e1, e2)


def test_autotuner_cache_on_the_device(Q, tmp_path):
    from paper_2406_17248_gb300 import tuning
    n = 16
    circ = I.random_circuit(n, 60, 5)
    s = Q.State(n, 0)
    path = str(tmp_path / "tune.json")
    c1, r1 = tuning.finalize_tuned(circ, 0, s, [], path)
    c2, r2 = tuning.finalize_tuned(circ, 0, s, [], path)
    assert not r1["cached"] and r2["cached"] and (r1["tile_bits"], r1["low_bits"]) == (r2["tile_bits"], r2["low_bits"])
    s.set_basis(0)
    c2.apply(s, [])
    assert np.abs(s.get_qs() - O.evolve(circ, [], O.zero_state(n))).max() < 5e-5
