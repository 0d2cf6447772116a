"""Variational training on the device: many independent (circuit, Hamiltonian,
parameters) instances -- for example the random starts of one DC-QAOA ansatz
(§5.4) -- optimised together with Adam, as the paper's training loops do with one
instance at a time (§4.1 gradient operator + an optimizer, §5.4 Adam on the
DC-QAOA cost F(alpha, beta, gamma)).

Each step is one batched energy + adjoint-gradient call (the persistent batched
kernel, replayed as a CUDA graph) and one Adam kernel over the concatenated
parameters; nothing goes to the host between steps.  PyTorch only holds the
device buffers."""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import inputs as I
from . import qsim as Q


class BatchAdam:
    """Minimise the energy of every instance with its own Adam state.

    instances: inputs.Instance list (their ``params`` are the starting points);
    dtype: qsim.C64 or qsim.C128.  After ``step()`` the tensors ``params``,
    ``energies`` (the energies at the parameters *before* the update) and
    ``grads`` live on the device."""

    def __init__(self, instances: Sequence[I.Instance], dtype: int = Q.C128, lr: float = 0.05,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        import torch
        self.batch = Q.Batch(list(instances), dtype)
        x0 = np.concatenate([np.asarray(it.params, dtype=np.float64) for it in instances])
        self.params = torch.tensor(x0, dtype=torch.float64, device="cuda")
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.energies = torch.zeros(len(instances), dtype=torch.float64, device="cuda")
        self.offsets = self.batch.param_offsets
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0

    def step(self):
        """One energy + gradient evaluation of every instance, then one Adam update."""
        self.batch.expectation_with_grad_device(self.params, self.energies, self.grads)
        self.t += 1
        Q.adam_f64(self.params, self.m, self.v, self.grads, self.t, self.lr, self.b1, self.b2, self.eps)

    def run(self, steps: int) -> np.ndarray:
        """``steps`` updates; returns the energy history, shape [steps, n_instances]."""
        import torch
        hist = torch.empty((steps, self.energies.numel()), dtype=torch.float64, device="cuda")
        for s in range(steps):
            self.step()
            hist[s].copy_(self.energies)
        return hist.cpu().numpy()

    def instance_params(self, i: int) -> np.ndarray:
        o = self.offsets
        return self.params[int(o[i]):int(o[i + 1])].cpu().numpy()


def dcqaoa_multistart(n: int, p: int, starts: int, seed: int, J: float = 1.0, h: float = 1.0, k: float = 0.0,
                      cd: bool = True, lo: float = 0.0, hi: float = 0.1):
    """``starts`` instances of the DC-QAOA ansatz on the Ising chain (§5.4), their
    starting parameters drawn U[lo, hi) from seeds seed, seed + 1, ..."""
    circ = I.dcqaoa_circuit(n, p, J, h, k, cd=cd)
    ham = I.lfim(n, J, h, k)
    return [I.Instance(circ, ham, I.uniform_params(circ.n_params, seed + s, lo, hi)) for s in range(starts)]


class GradientOperator:
    """The gradient operator of §4.1 with an encoder batch and a list of
    Hamiltonians: the circuit's parameters [0, n_encoder) are encoder inputs (one
    row per batch item) and the rest ansatz parameters shared by the batch.
    ``op(enc, ans)`` returns f [n_batch, n_ham], grad_enc [n_batch, n_ham,
    n_encoder] and grad_ans [n_batch, n_ham, n_ansatz] -- every (batch item,
    Hamiltonian) pair is one instance of a single batched launch (energy and
    adjoint gradient of each, in shared memory for small circuits)."""

    def __init__(self, circ: I.Circuit, hams: Sequence[I.PauliSum], n_encoder: int, n_batch: int,
                 dtype: int = Q.C128):
        if not 0 <= n_encoder <= circ.n_params:
            raise ValueError("n_encoder must be in [0, n_params]")
        self.n_enc, self.n_ans = n_encoder, circ.n_params - n_encoder
        self.n_batch, self.n_ham = n_batch, len(hams)
        zeros = np.zeros(circ.n_params)
        self.batch = Q.Batch([I.Instance(circ, h, zeros) for _ in range(n_batch) for h in hams], dtype)

    def __call__(self, enc, ans):
        enc = np.asarray(enc, dtype=np.float64).reshape(self.n_batch, self.n_enc)
        ans = np.asarray(ans, dtype=np.float64).reshape(self.n_ans)
        rows = np.concatenate([enc, np.broadcast_to(ans, (self.n_batch, self.n_ans))], axis=1)
        params = np.repeat(rows, self.n_ham, axis=0).reshape(-1)
        e, g = self.batch.expectation_with_grad(params)
        f = e.reshape(self.n_batch, self.n_ham)
        g = np.stack(g).reshape(self.n_batch, self.n_ham, self.n_enc + self.n_ans)
        return f, g[:, :, :self.n_enc], g[:, :, self.n_enc:]
