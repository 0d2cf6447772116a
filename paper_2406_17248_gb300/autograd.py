"""torch.autograd integration: the adjoint gradient becomes the backward pass.

The paper wraps its gradient operator as a trainable layer of a machine-learning
framework (MQLayer / MQAnsatzOnlyLayer, §4.1.2 and §5.2); here the same role is
played by torch.autograd.Function.  forward() makes ONE call of the engine,
which returns the energy and the full gradient (the adjoint sweep), keeps only
the gradient vector (p doubles) and returns the energy; backward() returns
dL/dE * grad without another simulation.  Parameters are FP64 host tensors
(the engine takes its angles on the host).
"""
from __future__ import annotations

from typing import Callable, Sequence, Tuple

import numpy as np
import torch

from . import inputs as I
from . import qsim as Q


class EnergyFunction(torch.autograd.Function):
    """E(params) with dE/dparams from an evaluator that returns both."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, evaluate: Callable[[np.ndarray], Tuple[float, np.ndarray]]):
        p = params.detach().to("cpu", torch.float64).numpy()
        energy, grad = evaluate(p)
        ctx.save_for_backward(torch.as_tensor(np.asarray(grad, dtype=np.float64)).to(params.device, params.dtype))
        return params.new_tensor(energy)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


class BatchEnergyFunction(torch.autograd.Function):
    """energies[i](params_i) for a batch, with the per-instance adjoint gradients."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, batch: "Q.Batch"):
        p = params.detach().to("cpu", torch.float64).numpy()
        e, grads = batch.expectation_with_grad(p)
        g = np.concatenate(grads) if grads else np.zeros(0)
        offs = torch.as_tensor(batch.param_offsets.astype(np.int64))
        ctx.save_for_backward(torch.as_tensor(g).to(params.device, params.dtype), offs)
        return params.new_tensor(e)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g, offs = ctx.saved_tensors
        counts = (offs[1:] - offs[:-1]).to(grad_out.device)
        scale = torch.repeat_interleave(grad_out, counts)
        return scale * g, None


class QAOAEnergy(torch.nn.Module):
    """MaxCut QAOA energy <C> as a module with trainable gamma and beta (§5.2)."""

    def __init__(self, n: int, edges, p: int, gamma_scale: float = 0.5, dtype: int = Q.C64,
                 gamma0=None, beta0=None):
        super().__init__()
        self.p = p
        self.engine = Q.QAOA(n, edges, p, gamma_scale=gamma_scale, dtype=dtype)
        self.psi, self.lam = Q.State(n, dtype), Q.State(n, dtype)
        g0 = np.zeros(p) if gamma0 is None else np.asarray(gamma0, dtype=np.float64)
        b0 = np.zeros(p) if beta0 is None else np.asarray(beta0, dtype=np.float64)
        self.gamma = torch.nn.Parameter(torch.tensor(g0, dtype=torch.float64))
        self.beta = torch.nn.Parameter(torch.tensor(b0, dtype=torch.float64))

    def _evaluate(self, x: np.ndarray):
        e, dg, db = self.engine.expectation_with_grad(self.psi, self.lam, x[: self.p], x[self.p:])
        return e, np.concatenate([dg, db])

    def forward(self) -> torch.Tensor:
        return EnergyFunction.apply(torch.cat([self.gamma, self.beta]), self._evaluate)


class CircuitEnergy(torch.nn.Module):
    """<psi(params)|H|psi(params)> of a parameterised circuit from a fixed start state."""

    def __init__(self, circuit: I.Circuit, ham: I.PauliSum, dtype: int = Q.C64, params0=None, psi0=None):
        super().__init__()
        n = circuit.n_qubits
        self.circuit = Q.circuit_from(circuit).finalize(dtype)
        self.ham = Q.Hamiltonian(ham)
        self.psi, self.lam = Q.State(n, dtype), Q.State(n, dtype)
        self._psi0 = None if psi0 is None else np.asarray(psi0)
        p0 = np.zeros(circuit.n_params) if params0 is None else np.asarray(params0, dtype=np.float64)
        self.params = torch.nn.Parameter(torch.tensor(p0, dtype=torch.float64))

    def _evaluate(self, x: np.ndarray):
        if self._psi0 is None:
            self.psi.set_basis(0)
        else:
            self.psi.set_qs(self._psi0)
        return Q.expectation_with_grad(self.psi, self.lam, self.circuit, self.ham, x)

    def forward(self) -> torch.Tensor:
        return EnergyFunction.apply(self.params, self._evaluate)


class BatchEnergy(torch.nn.Module):
    """Energies of a batch of independent instances (one persistent launch per call)."""

    def __init__(self, instances: Sequence[I.Instance], dtype: int = Q.C64):
        super().__init__()
        self.batch = Q.Batch(list(instances), dtype)
        p0 = np.concatenate([np.asarray(it.params, dtype=np.float64) for it in instances])
        self.params = torch.nn.Parameter(torch.tensor(p0, dtype=torch.float64))

    def forward(self) -> torch.Tensor:
        return BatchEnergyFunction.apply(self.params, self.batch)
