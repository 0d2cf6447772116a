"""The C-ABI library builds, loads and exports every entry point include/qsim.h
declares; host-side argument checks reject bad input before any device work."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_2406_17248_gb300 import build as B
from paper_2406_17248_gb300 import qsim as Q

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "qsim.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^QS_API\s+[\w\s\*]+?\b(qs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return Q.lib()


def test_header_declares_the_binding_signatures():
    assert declared_symbols() == sorted(n for n, _ in Q.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version_string(lib):
    assert b"sm_103a" in lib.qs_version()


def test_circuit_argument_checks_run_on_the_host(lib):
    c = Q.Circuit(3)
    with pytest.raises(Q.QSimError, match="out of range"):
        c.add("X", [3])
    with pytest.raises(Q.QSimError, match="repeats"):
        c.add("X", [0], [0])
    with pytest.raises(Q.QSimError, match="wrong number of targets"):
        c.add("RZZ", [0])
    with pytest.raises(Q.QSimError, match="only RX"):
        c.add("H", [0], param=0)
    with pytest.raises(Q.QSimError, match="MATRIX gate needs"):
        c.add("MATRIX", [0])
    c.add("RX", [0], [1], param=2)
    assert c.info()["params"] == 3 and c.info()["gates"] == 1
    h = C.c_void_p()
    assert lib.qs_circuit_create(0, C.byref(h)) == 1
    assert lib.qs_circuit_create(35, C.byref(h)) == 1


def test_qaoa_argument_checks_run_on_the_host(lib):
    with pytest.raises(Q.QSimError, match="self-loop"):
        Q.QAOA(5, [(0, 0)], 1)
    with pytest.raises(Q.QSimError, match="repeated edge"):
        Q.QAOA(5, [(0, 1), (1, 0)], 1)
    with pytest.raises(Q.QSimError, match="n_qubits"):
        Q.QAOA(3, [(0, 1)], 1)
    with pytest.raises(Q.QSimError, match="p must be"):
        Q.QAOA(5, [(0, 1)], 0)


def test_null_handles_are_rejected(lib):
    v = C.c_double()
    assert lib.qs_state_norm2(None, C.byref(v)) == 1
    assert lib.qs_expectation(None, None, C.byref(v)) == 1
    assert b"null" in lib.qs_last_error()


def test_trajectory_argument_checks_run_on_the_host(lib):
    h = C.c_void_p()
    assert lib.qs_traj_create(35, 0, None, C.byref(h)) == 1
    assert b"1..34" in lib.qs_last_error()
    assert lib.qs_traj_create(3, 0, None, C.byref(h)) == 0
    t = (C.c_int * 1)(3)
    assert lib.qs_traj_add_gate(h, Q.KIND["X"], t, 1, None, 0, -1, 1.0, 0.0) == 1
    assert b"out of range" in lib.qs_last_error()
    t[0] = 0
    assert lib.qs_traj_add_gate(h, Q.KIND["MATRIX"], t, 1, None, 0, -1, 1.0, 0.0) == 1

    def chan(kind, q, p, kraus=None):
        pr = np.ascontiguousarray(p if len(p) else [0.0], dtype=np.float64)
        kr = None if kraus is None else np.ascontiguousarray(np.asarray(kraus, dtype=np.complex128)).view(np.float64)
        return lib.qs_traj_add_channel(h, Q.CHANNELS[kind], q, pr.ctypes.data_as(Q._PD), 0 if kraus is None else len(kraus),
                                       None if kr is None else kr.ctypes.data_as(Q._PD))

    assert chan("pauli", 0, (0.5, 0.4, 0.2)) == 1 and b"sum <= 1" in lib.qs_last_error()
    assert chan("amplitude_damping", 0, (1.5,)) == 1 and b"gamma" in lib.qs_last_error()
    assert chan("kraus", 1, (), [np.eye(2) * 0.5]) == 1 and b"not complete" in lib.qs_last_error()
    assert chan("kraus", 1, (), [np.eye(2) / math.sqrt(5)] * 5) == 1 and b"1..4 Kraus" in lib.qs_last_error()
    assert lib.qs_traj_add_gate(h, Q.KIND["RX"], t, 1, None, 0, 1, 1.0, 0.0) == 0
    assert chan("depolarizing", 2, (0.1,)) == 0
    assert chan("kraus", 1, (), [np.eye(2) / math.sqrt(2)] * 2) == 0
    a, b = C.c_int(), C.c_int()
    assert lib.qs_traj_info(h, C.byref(a), C.byref(b), None, None) == 0
    assert (a.value, b.value) == (2, 2)
    lib.qs_traj_destroy(h)
