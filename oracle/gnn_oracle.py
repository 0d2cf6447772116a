"""FP64 CPU oracle of the learned QAOA initialiser (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm may import this module; the product never calls it and shares no
code with it.

The paper trains QAOA angles by gradient descent from a fixed start (§5.2:
the MindSpore optimiser drives the ansatz parameters) and motivates a slowly
varying schedule by the adiabatic picture (§5.4, DC-QAOA background).
It does not define a learned initialiser; the network below is this project's
definition, stated once here and once in the CUDA library:

* input: an undirected graph, node features h0[v] = (1, deg(v) / 3).
* L message-passing layers of width H:
      a[v]   = mean of h[u] over the neighbours u of v (0 if v has none)
      h'[v]  = relu(Ws h[v] + Wn a[v] + b)
* readout r = mean of h_L[v] over the nodes (0 for an empty graph),
  z = relu(W1 r + b1), y = W2 z + b2: the 2p angles (gamma_1..p, beta_1..p).
* parameters: one flat vector, per layer Ws [H x d], Wn [H x d], b [H]
  (d = 2 for the first layer, H after), then W1 [H x H], b1 [H], W2 [O x H],
  b2 [O]; matrices row-major (output, input).
* the network computes with weights rounded to bfloat16 (round to nearest,
  ties to even); this oracle takes those rounded values and does everything
  else in float64.
* loss: mean squared error over graphs and outputs.
* optimiser: Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.

Parity: the forward pass is pinned by permutation invariance, by the reduction
of a regular graph with equal node features to a plain MLP, and by the empty
and edgeless graphs; the backward pass by central finite differences of the
forward; bfloat16 rounding by exact values; Adam by its first step
(lr * sign(g) up to eps) and a hand-run two-step sequence (tests/test_gnn_oracle.py).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def layout(hidden: int = 64, layers: int = 3, out_dim: int = 8, in_dim: int = 2) -> List[Tuple[str, str, int, int]]:
    """[(name, kind, rows, cols)] blocks of the flat parameter vector, in order."""
    out = []
    d = in_dim
    for l in range(layers):
        out += [(f"Ws{l}", "W", hidden, d), (f"Wn{l}", "W", hidden, d), (f"bl{l}", "b", hidden, 1)]
        d = hidden
    out += [("W1", "W", hidden, hidden), ("b1", "b", hidden, 1), ("W2", "W", out_dim, hidden), ("b2", "b", out_dim, 1)]
    return out


def n_weights(**dims) -> int:
    return sum(r * c for _, _, r, c in layout(**dims))


def unpack(w: np.ndarray, **dims) -> Dict[str, np.ndarray]:
    """Views of the flat vector as named float64 matrices / vectors."""
    out, o = {}, 0
    for name, kind, r, c in layout(**dims):
        blk = np.asarray(w[o:o + r * c], dtype=np.float64)
        out[name] = blk.reshape(r, c) if kind == "W" else blk
        o += r * c
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 values rounded to bfloat16 (8 exponent, 7 mantissa bits), round to
    nearest with ties to even, returned as float64.  Finite inputs only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _graph_lists(node_off, adj_off, adj):
    """[(n_nodes, neighbour lists)] per graph from the CSR batch."""
    out = []
    for g in range(len(node_off) - 1):
        v0, v1 = int(node_off[g]), int(node_off[g + 1])
        nb = [[int(u) for u in adj[adj_off[v]:adj_off[v + 1]]] for v in range(v0, v1)]
        out.append((v1 - v0, nb))
    return out


def _forward_graph(P, n, nb, layers):
    """Per-layer activations of one graph: (h list, a list, r, zpre, y)."""
    deg = np.array([len(x) for x in nb], dtype=np.float64)
    h = np.stack([np.ones(n), deg / 3.0], axis=1) if n else np.zeros((0, 2))
    hs, as_ = [h], []
    for l in range(layers):
        a = np.zeros_like(h)
        for v in range(n):
            if nb[v]:
                a[v] = h[nb[v]].mean(axis=0)
        pre = h @ P[f"Ws{l}"].T + a @ P[f"Wn{l}"].T + P[f"bl{l}"]
        h = np.maximum(pre, 0.0)
        as_.append(a)
        hs.append(h)
    r = h.mean(axis=0) if n else np.zeros(P["W1"].shape[1])
    zpre = P["W1"] @ r + P["b1"]
    z = np.maximum(zpre, 0.0)
    y = P["W2"] @ z + P["b2"]
    return hs, as_, r, zpre, y


def forward(w_bf16: np.ndarray, node_off, adj_off, adj, layers: int = 3, **dims) -> np.ndarray:
    """y[G, O] for every graph of the batch; w_bf16 holds the bfloat16-rounded
    weights (float64 values)."""
    P = unpack(w_bf16, layers=layers, **dims)
    return np.array([_forward_graph(P, n, nb, layers)[4] for n, nb in _graph_lists(node_off, adj_off, adj)])


def mse(y: np.ndarray, t: np.ndarray) -> Tuple[float, np.ndarray]:
    """(loss, dloss/dy) of the mean squared error over all entries."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(w_bf16: np.ndarray, node_off, adj_off, adj, dy: np.ndarray, layers: int = 3, **dims) -> np.ndarray:
    """dL/dw (flat, same layout) given dL/dy[G, O], by reverse-mode chain rule."""
    P = unpack(w_bf16, layers=layers, **dims)
    G = {k: np.zeros_like(v) for k, v in P.items()}
    for gi, (n, nb) in enumerate(_graph_lists(node_off, adj_off, adj)):
        hs, as_, r, zpre, y = _forward_graph(P, n, nb, layers)
        z = np.maximum(zpre, 0.0)
        g_y = dy[gi]
        G["W2"] += np.outer(g_y, z)
        G["b2"] += g_y
        g_zpre = (P["W2"].T @ g_y) * (zpre > 0)
        G["W1"] += np.outer(g_zpre, r)
        G["b1"] += g_zpre
        g_r = P["W1"].T @ g_zpre
        g_h = np.tile(g_r / n, (n, 1)) if n else np.zeros((0, g_r.size))
        for l in range(layers - 1, -1, -1):
            g_pre = g_h * (hs[l + 1] > 0)
            G[f"Ws{l}"] += g_pre.T @ hs[l]
            G[f"Wn{l}"] += g_pre.T @ as_[l]
            G[f"bl{l}"] += g_pre.sum(axis=0)
            g_a = g_pre @ P[f"Wn{l}"]
            g_hl = g_pre @ P[f"Ws{l}"]
            for v in range(n):
                if nb[v]:
                    for u in nb[v]:
                        g_hl[u] += g_a[v] / len(nb[v])
            g_h = g_hl
    return np.concatenate([G[name].reshape(-1) for name, _, _, _ in layout(layers=layers, **dims)])


def adam(w, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (t = 1, 2, ...): returns new (w, m, v) in float64."""
    w, m, v, g = (np.asarray(x, dtype=np.float64) for x in (w, m, v, g))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def min_abs_preactivation(w_bf16: np.ndarray, node_off, adj_off, adj, layers: int = 3, **dims) -> float:
    """Smallest |pre-activation| of any ReLU in the batch (message-passing layers
    and the readout MLP).  Tests use it to keep inputs away from the kink, where
    float32 and float64 may take different branches of the derivative."""
    P = unpack(w_bf16, layers=layers, **dims)
    best = np.inf
    for n, nb in _graph_lists(node_off, adj_off, adj):
        hs, as_, r, zpre, y = _forward_graph(P, n, nb, layers)
        for l in range(layers):
            if n:
                pre = hs[l] @ P[f"Ws{l}"].T + as_[l] @ P[f"Wn{l}"].T + P[f"bl{l}"]
                best = min(best, float(np.min(np.abs(pre))))
        best = min(best, float(np.min(np.abs(zpre))))
    return best
