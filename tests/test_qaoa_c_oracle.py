"""Pins of the C FP64 QAOA oracle (oracle/qaoa_oracle.c), which times the CPU
baseline: the printed QuPack K5 values (§6.2.2), the gamma = 0 closed form,
central finite differences, agreement with the numpy oracle, and independence
of the thread count."""
import json
import os

import numpy as np
import pytest

from oracle import qaoa_c
from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_printed_qupack_k5_values():
    g = json.load(open(os.path.join(GOLD, "qupack_qaoa_k5.json")))
    n, p = g["n_qubits"], g["depth"]
    E, dg, db = qaoa_c.evaluate(n, I.complete_graph(n), [g["gamma"]] * p, [g["beta"]] * p, 1.0)
    assert abs(E - g["expectation"]) < 1e-12
    np.testing.assert_allclose(dg, g["gamma_grad"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(db, g["beta_grad"], rtol=0, atol=1e-10)


def test_gamma_zero_closed_form():
    """RX on every qubit maps |+>^n to a phase times itself, and <+|z_a z_b|+> = 0:
    E = 0 and dE/dbeta = 0 whatever beta."""
    n = 9
    edges = I.random_regular_graph(n - 1, 3, 2)
    E, dg, db = qaoa_c.evaluate(n, edges, [0.0] * 3, [0.3, 1.7, 2.9], 0.5)
    assert abs(E) < 1e-13 and np.abs(db).max() < 1e-12


def test_central_differences():
    n, p = 8, 3
    edges = I.random_regular_graph(n, 3, 4)
    ang = I.uniform_params(2 * p, 11, 0.0, np.pi)
    g, b = ang[:p], ang[p:]
    E, dg, db = qaoa_c.evaluate(n, edges, g, b, 0.5)
    h = 1e-5
    for k in range(p):
        for arr, grad in ((g, dg), (b, db)):
            up, dn = arr.copy(), arr.copy()
            up[k] += h
            dn[k] -= h
            args_up = (up, b) if arr is g else (g, up)
            args_dn = (dn, b) if arr is g else (g, dn)
            fd = (qaoa_c.evaluate(n, edges, *args_up, 0.5)[0] - qaoa_c.evaluate(n, edges, *args_dn, 0.5)[0]) / (2 * h)
            assert abs(fd - grad[k]) < 1e-7


@pytest.mark.parametrize("n,p,gs", [(10, 4, 0.5), (11, 2, 1.0)])
def test_agrees_with_numpy_oracle_at_any_thread_count(n, p, gs):
    edges = I.random_regular_graph(n, 3 if n % 2 == 0 else 4, 7)
    ang = I.uniform_params(2 * p, n, 0.0, np.pi)
    E0, dg0, db0 = O.qaoa_expectation_with_grad(n, edges, ang[:p], ang[p:], gs)
    for th in (1, 3):
        E, dg, db = qaoa_c.evaluate(n, edges, ang[:p], ang[p:], gs, threads=th)
        assert abs(E - E0) < 1e-12
        assert np.abs(dg - dg0).max() < 1e-11 and np.abs(db - db0).max() < 1e-11
