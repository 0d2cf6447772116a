"""The C-ABI library builds, loads and exports every entry point include/qsim.h
declares; host-side argument checks reject bad input before any device work."""
import ctypes as C
import os
import re

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
