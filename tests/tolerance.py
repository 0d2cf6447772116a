"""One tolerance rule for every GPU parity result, and a record of the errors seen.

The stated accuracy is a max-abs amplitude error of tol = 1e-11 (complex128) or
5e-5 (complex64).  Every other result is held to tol times the largest magnitude
that result can take, so the same relative accuracy applies to each:

* amplitudes of an evolved state: tol (max-abs).  For whole states the tests
  check the 2-norm of the error, ||psi - psi_ref||_2 <= tol, which implies the
  max-abs bound and stays meaningful at large n where every amplitude is far
  below tol.  A sampled amplitude of an n-qubit state is held to tol * 2^(-n/2),
  its share of that 2-norm when the error is spread over the state.
* a state returned to its start by the reverse sweep or by a circuit and its
  inverse passes through twice the gate applications of one evolution: 2 tol.
  Its norm then differs from 1 by at most 2 ||delta|| + ||delta||^2.
* energy <psi|H|psi> of H = sum_k c_k P_k: |E| <= sum_k |c_k|, so the bound is
  tol * max(1, sum_k |c_k|).
* gradient dE/dp = sum over the gates k bound to p of coef_k g_k, with
  g_k = 2 Re <lam| dU_k/dtheta |psi> and |g_k| <= 2 ||dU_k/dtheta|| ||H|| (the
  adjoint method, §4.1).  For R_P(theta) = exp(-i theta P / 2) (RX, RY, RZ, RXX,
  RYY, RZZ, with or without controls) ||dU/dtheta|| = 1/2; for PhaseShift
  diag(1, e^{i theta}) it is 1.  So |dE/dp| <= sum_k w_k |coef_k| * sum |c|
  (w = 1 for R_P, 2 for PhaseShift), and the bound is
  tol * max(1, sum |c|) * max(1, sum_k w_k |coef_k|).  A QAOA parameter is shared
  by many gates: gamma_l by |E| RZZ(2 gs gamma_l) gates (coef 2 gs each), beta_l
  by n RX(beta_l) gates.

``check`` asserts err <= bound and records (test, result, err, bound); the
session writes the records as JSON to the path in QS_ERR_LOG when it is set, so
the measured errors can be stated per result.
"""
import json
import os

import numpy as np

TOL = {0: 5e-5, 1: 1e-11}

_RECORDS = []


def ham_scale(ham) -> float:
    """max(1, sum |c_k|): the bound on |<psi|H|psi>| for a normalised psi."""
    return max(1.0, float(np.abs(np.asarray(ham.coef)).sum()))


def energy_tol(dt: int, ham) -> float:
    return TOL[dt] * ham_scale(ham)


_W = {"RX": 1.0, "RY": 1.0, "RZ": 1.0, "RXX": 1.0, "RYY": 1.0, "RZZ": 1.0, "PS": 2.0}


def param_bound(circ) -> np.ndarray:
    """Per parameter p: max(1, sum over gates bound to p of w_k |coef_k|)."""
    b = np.zeros(max(1, circ.n_params))
    for g in circ.gates:
        if g.param >= 0:
            b[g.param] += _W.get(g.kind, 2.0) * abs(g.coef)
    return np.maximum(1.0, b[: circ.n_params])


def grad_tol(dt: int, ham, circ) -> np.ndarray:
    """Per-parameter gradient bound for a circuit (see the module docstring)."""
    return TOL[dt] * ham_scale(ham) * param_bound(circ)


def qaoa_grad_tols(dt: int, n: int, n_edges: int, gamma_scale: float):
    """(energy, dgamma_l, dbeta_l) bounds of a MaxCut QAOA layer: the cost
    exp(-i gs gamma C) = prod over edges RZZ(2 gs gamma), the mixer RX(beta) per qubit."""
    e = TOL[dt] * max(1.0, n_edges)
    return e, e * max(1.0, 2.0 * abs(gamma_scale) * n_edges), e * max(1.0, n)


def state_err(got, want) -> float:
    """||got - want||_2 (the 2-norm of the amplitude error)."""
    d = np.asarray(got, dtype=np.complex128) - np.asarray(want, dtype=np.complex128)
    return float(np.sqrt(np.sum(d.real ** 2 + d.imag ** 2)))


def check(name: str, err, bound) -> None:
    """Assert err <= bound elementwise and record the worst ratio."""
    err = np.atleast_1d(np.asarray(err, dtype=np.float64))
    bound = np.broadcast_to(np.atleast_1d(np.asarray(bound, dtype=np.float64)), err.shape)
    ratio = err / bound
    i = int(np.argmax(ratio)) if err.size else 0
    _RECORDS.append({"name": name, "err": float(err[i]) if err.size else 0.0,
                     "bound": float(bound[i]) if err.size else 0.0,
                     "ratio": float(ratio[i]) if err.size else 0.0})
    assert np.all(err <= bound), f"{name}: error {err[i]:.3e} above its bound {bound[i]:.3e}"


def write_records() -> None:
    path = os.environ.get("QS_ERR_LOG")
    if not path or not _RECORDS:
        return
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(_RECORDS, f, indent=0)
