"""Loader of the C FP64 QAOA oracle (qaoa_oracle.c) -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__`` (build and smoke) and ``bench.py``'s CPU
baseline and reference arm may import this module.  ``build()`` compiles the C
source with the host gcc (OpenMP on, no machine-specific flags) into
oracle/_build/; ``evaluate()`` runs one energy + adjoint-gradient evaluation
(§6.2 QuPack QAOA, §4.1 adjoint method) on ``threads`` host threads.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qaoa_oracle.c")
OUT = os.path.join(HERE, "_build", "libqaoa_oracle.so")
_lib = None


def build() -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, OUT)
    return OUT


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.qaoa_oracle_eval.restype = C.c_int
        _lib.qaoa_oracle_eval.argtypes = [C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.c_double, C.c_int, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib.qaoa_oracle_max_threads.restype = C.c_int
    return _lib


def max_threads() -> int:
    return int(lib().qaoa_oracle_max_threads())


def evaluate(n: int, edges, gamma, beta, gamma_scale: float = 1.0, threads: int = 0):
    """(E, dE/dgamma[p], dE/dbeta[p]) in FP64."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    p = int(g.size)
    assert b.size == p
    E = C.c_double()
    dg = np.zeros(p)
    db = np.zeros(p)
    dp = C.POINTER(C.c_double)
    rc = lib().qaoa_oracle_eval(n, e.ctypes.data_as(C.POINTER(C.c_int)), int(e.size // 2), p, g.ctypes.data_as(dp),
                                b.ctypes.data_as(dp), float(gamma_scale), int(threads), C.byref(E),
                                dg.ctypes.data_as(dp), db.ctypes.data_as(dp))
    if rc != 0:
        raise ValueError("qaoa_oracle_eval: bad arguments or out of host memory")
    return E.value, dg, db
