"""Learned QAOA initialiser: a graph network predicts the 2p angles of MaxCut
QAOA from the graph; it is trained on angles the simulator optimised.

The paper trains QAOA angles by gradient descent from a fixed start (§5.2) and
motivates slowly varying schedules by adiabatic evolution (§5.4).  This module
supplies the pieces around the CUDA kernels (qs_gnn_*, qs_batch_*, qs_adam_f64):

* linear_ramp: the adiabatic-style baseline start.
* canonicalise: one representative of each class of angles with equal energy.
* AngleOptimiser: Adam on the angles of many QAOA instances at once -- one
  batched energy+gradient launch and one Adam launch per step, on the device.
* Initialiser: the network, its training loop (one fused training-step launch
  plus the gradient-sum/Adam launch per batch) and prediction.
* steps_to_ratio: Adam steps until the approximation ratio reaches a target.

Angle convention (the circuit of §5.2): layer l applies RZZ(g_l) on every edge,
RZZ(t) = exp(-i t/2 Z Z), then RX(b_l) on every qubit; the vector is
[g_1..g_p, b_1..b_p].  The energy is <sum over edges of Z_a Z_b>, which the
optimiser minimises; the expected cut is (|E| - energy) / 2.
"""
from __future__ import annotations

import math
import time
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import inputs as I
from . import qsim as Q

Graph = Tuple[int, Sequence[Tuple[int, int]]]


def linear_ramp(p: int, delta: float = 0.75) -> np.ndarray:
    """Trotterised adiabatic path from |+>^n, the ground state of -sum X, to the
    ground state of sum ZZ: layer l runs exp(-i gamma_l sum ZZ) exp(+i beta_l sum X)
    with gamma_l = (l - 1/2)/p * delta and beta_l = (1 - (l - 1/2)/p) * delta, i.e.
    gate angles g_l = 2 gamma_l and b_l = -2 beta_l."""
    s = (np.arange(1, p + 1) - 0.5) / p
    return np.concatenate([2.0 * s * delta, -2.0 * (1.0 - s) * delta])


def canonicalise(angles: np.ndarray, p: int) -> np.ndarray:
    """Representative of the angles' symmetry class.  The energy is unchanged by
    g_l -> g_l + 2 pi (the cost's eigenvalues share the parity of |E|, so the
    shift is a global phase), by b_l -> b_l + pi (RX(b + pi) = -i X RX(b) and
    the global flip X^n commutes with the circuit, fixes |+>^n and the cost),
    and by negating every angle (complex conjugation of a real-start circuit).
    Result: b in [-pi/2, pi/2), g in [-pi, pi) with g_1 >= 0."""
    a = np.array(angles, dtype=np.float64, copy=True).reshape(-1, 2 * p)

    def wrap(x):
        x[:, :p] = (x[:, :p] + math.pi) % (2 * math.pi) - math.pi
        x[:, p:] = (x[:, p:] + math.pi / 2) % math.pi - math.pi / 2
        return x

    a = wrap(a)
    neg = a[:, 0] < 0
    a[neg] = wrap(-a[neg])
    return a.reshape(np.shape(angles))


def qaoa_instance(n: int, edges, p: int) -> I.Instance:
    return I.Instance(I.qaoa_circuit(n, edges, p, gamma_coef=1.0), I.maxcut_zz(n, edges), np.zeros(2 * p))


class AngleOptimiser:
    """Adam on the angles of a list of QAOA instances (graph, p), all at once."""

    def __init__(self, graphs: Sequence[Graph], p: int, dtype: int = Q.C64, stream=None):
        import torch
        self.graphs, self.p = list(graphs), p
        self.stream = stream
        self.batch = Q.Batch([qaoa_instance(n, e, p) for n, e in self.graphs], dtype, stream)
        self.n_inst = len(self.graphs)
        dev = torch.device("cuda")
        self._t = lambda *shape: torch.zeros(*shape, dtype=torch.float64, device=dev)

    def run(self, init: np.ndarray, steps: int, lr: float = 0.05, record: bool = True):
        """Run `steps` Adam steps from init[n_inst, 2p].  Returns (final angles,
        energies[steps + 1, n_inst] (row t: before step t+1; last row: final angles)
        or only the last row when record is False, seconds)."""
        import torch
        k = self.n_inst * 2 * self.p
        params = torch.as_tensor(np.ascontiguousarray(init, dtype=np.float64).reshape(-1)).cuda()
        m, v, g = self._t(k), self._t(k), self._t(k)
        hist = self._t(steps + 1 if record else 1, self.n_inst)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(steps):
            row = hist[t] if record else hist[0]
            self.batch.expectation_with_grad_device(params, row, g)
            Q.adam_f64(params, m, v, g, t + 1, lr, stream=self.stream)
        self.batch.expectation_with_grad_device(params, hist[-1], g)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return params.view(self.n_inst, 2 * self.p).cpu().numpy(), hist.cpu().numpy(), dt


def optimised_angles(graphs: Sequence[Graph], p: int, restarts: int = 4, steps: int = 200, lr: float = 0.05,
                     seed: int = 0, delta: float = 0.75, chunk: int = 4096):
    """Labels for training: Adam from the linear ramp and from `restarts` uniform
    random starts per graph; the best final energy wins.  Returns (canonical
    angles[G, 2p], best energies[G])."""
    rng = np.random.default_rng(seed)
    G = len(graphs)
    starts = [np.tile(linear_ramp(p, delta), (G, 1))]
    for _ in range(restarts):
        starts.append(np.concatenate([rng.uniform(-math.pi, math.pi, (G, p)),
                                      rng.uniform(-math.pi / 2, math.pi / 2, (G, p))], axis=1))
    best = np.full(G, np.inf)
    best_a = np.zeros((G, 2 * p))
    for c0 in range(0, G, chunk):
        sub = list(graphs[c0:c0 + chunk])
        inst = sub * len(starts)
        init = np.concatenate([s[c0:c0 + len(sub)] for s in starts])
        final, hist, _ = AngleOptimiser(inst, p).run(init, steps, lr, record=False)
        e = hist[-1].reshape(len(starts), len(sub))
        a = final.reshape(len(starts), len(sub), 2 * p)
        k = np.argmin(e, axis=0)
        idx = np.arange(len(sub))
        best[c0:c0 + len(sub)] = e[k, idx]
        best_a[c0:c0 + len(sub)] = a[k, idx]
    return canonicalise(best_a, p), best


class Initialiser:
    """The graph network (qs_gnn_*) mapping a graph to 2p angles."""

    def __init__(self, p: int = 4, hidden: int = 64, layers: int = 3, seed: int = 0, stream=None):
        self.p = p
        self.stream = stream
        self.net = Q.GNN(hidden, layers, 2 * p, stream)
        lay = []
        d = 2
        for _ in range(layers):
            lay += [("W", hidden, d), ("W", hidden, d), ("b", hidden, 1)]
            d = hidden
        lay += [("W", hidden, hidden), ("b", hidden, 1), ("W", 2 * p, hidden), ("b", 2 * p, 1)]
        self.net.set_weights(I.gnn_init_weights(lay, seed))

    def fit(self, graphs: Sequence[Graph], targets: np.ndarray, epochs: int = 50, batch_size: int = 256,
            lr: float = 1e-3, seed: int = 0, log_every: int = 0):
        """Minimise the MSE to targets[G, 2p]; returns the mean loss per epoch."""
        import torch
        dev = torch.device("cuda")
        rng = np.random.default_rng(seed)
        order = rng.permutation(len(graphs))
        batches = []
        for b0 in range(0, len(graphs), batch_size):
            idx = order[b0:b0 + batch_size]
            gb = Q.Graphs.from_graphs([graphs[i] for i in idx])
            tb = torch.as_tensor(np.asarray(targets, dtype=np.float32)[idx]).to(dev)
            batches.append((gb, tb))
        losses = torch.zeros(epochs, len(batches), dtype=torch.float32, device=dev)
        for ep in range(epochs):
            for bi in rng.permutation(len(batches)):
                gb, tb = batches[bi]
                self.net.train_step(gb, tb, lr, losses[ep, bi:bi + 1])
            if log_every and (ep + 1) % log_every == 0:
                print(f"epoch {ep + 1}: loss {losses[ep].mean().item():.5f}", flush=True)
        return losses.mean(dim=1).cpu().numpy()

    def predict(self, graphs: Sequence[Graph]) -> np.ndarray:
        import torch
        gb = Q.Graphs.from_graphs(graphs)
        y = torch.zeros(len(graphs), 2 * self.p, dtype=torch.float32, device="cuda")
        self.net.forward(gb, y)
        return y.cpu().numpy().astype(np.float64)


def max_cuts(graphs: Sequence[Graph]) -> np.ndarray:
    """Exact MaxCut of every graph (exhaustive search on the device).  Graphs
    below 4 nodes are padded with isolated nodes, which leave the cut unchanged;
    a graph without edges has MaxCut 0."""
    out = []
    for n, e in graphs:
        if len(e) == 0:
            out.append(0)
            continue
        q = Q.QAOA(max(n, 4), e, 1, 0.5)
        out.append(q.max_cut())
        q.close()
    return np.array(out, dtype=np.float64)


def _adam_on_engine(q, n: int, init: np.ndarray, p: int, steps: int, lr: float):
    """Adam on one graph through the QAOA engine (energy and adjoint gradient),
    with the Adam update done by the device kernel.  Returns energies[steps + 1]."""
    import torch
    psi, lam = Q.State(n), Q.State(n)
    w = torch.as_tensor(np.array(init, dtype=np.float64)).cuda()
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    e = np.zeros(steps + 1)
    a = np.array(init, dtype=np.float64)
    for t in range(steps + 1):
        E, dg, db = q.expectation_with_grad(psi, lam, a[:p], a[p:])
        e[t] = E
        if t == steps:
            break
        Q.adam_f64(w, m, v, torch.as_tensor(np.concatenate([dg, db])).cuda(), t + 1, lr)
        a = w.cpu().numpy()
    return e


def steps_to_ratio(graphs: Sequence[Graph], init: np.ndarray, p: int, steps: int = 200, lr: float = 0.05,
                   target: float = 0.9, maxcut: Optional[np.ndarray] = None, engine: str = "auto"):
    """Adam from init[G, 2p] for every graph; the approximation ratio of step t is
    (|E| - E_t) / 2 / maxcut.  engine: "batch" (all graphs in one persistent
    launch per step; fastest while states fit in shared memory, n <= 13), "qaoa"
    (the fused-pass QAOA engine, graph by graph) or "auto".  Returns (steps to
    reach `target` per graph, -1 where not reached; ratio trajectories
    [steps + 1, G]; seconds)."""
    import torch
    mc = max_cuts(graphs) if maxcut is None else np.asarray(maxcut, dtype=np.float64)
    ne = np.array([len(e) for _, e in graphs], dtype=np.float64)
    if engine == "auto":
        engine = "batch" if max(n for n, _ in graphs) <= 13 else "qaoa"
    if engine == "batch":
        _, hist, dt = AngleOptimiser(graphs, p).run(init, steps, lr, record=True)
    else:
        hist = np.zeros((steps + 1, len(graphs)))
        dt = 0.0
        for i, (n, e) in enumerate(graphs):
            q = Q.QAOA(max(n, 4), e, p, 0.5)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hist[:, i] = _adam_on_engine(q, max(n, 4), init[i], p, steps, lr)
            torch.cuda.synchronize()
            dt += time.perf_counter() - t0
            q.close()
    ratio = (ne[None, :] - hist) / 2.0 / mc[None, :]
    hit = ratio >= target
    first = np.where(hit.any(axis=0), hit.argmax(axis=0), -1)
    return first, ratio, dt
