"""Pins of the FP64 GNN oracle (learned QAOA initialiser): exact bfloat16
values, graph symmetries and special cases that reduce the network to a plain
MLP, finite differences for the backward pass, and Adam's textbook first steps."""
import numpy as np
import pytest

from oracle import gnn_oracle as G
from paper_2406_17248_gb300 import inputs as I

SMALL = dict(hidden=8, layers=2, out_dim=4)


def _weights(seed, **dims):
    lay = [(k, r, c) for _, k, r, c in G.layout(**dims)]
    w = I.gnn_init_weights(lay, seed).astype(np.float64)
    # non-zero biases so that every term of the network is exercised
    rng = np.random.default_rng(seed + 1)
    o = 0
    for _, k, r, c in G.layout(**dims):
        if k == "b":
            w[o:o + r] = rng.uniform(-0.3, 0.3, size=r)
        o += r * c
    return G.bf16_round(w)


def test_bf16_round_exact_values():
    x = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-8, -(1 + 2**-7), 3.0, 1.0 / 3.0, 0.0, -2.5], dtype=np.float32)
    want = [1.0, 1.0, 1 + 2**-6, -(1 + 2**-7), 3.0, 0.333984375, 0.0, -2.5]
    assert G.bf16_round(x).tolist() == want


def test_layout_size_closed_form():
    # per layer 2*H*d + H, then H*H + H + O*H + O
    assert G.n_weights() == (2 * 64 * 2 + 64) + 2 * (2 * 64 * 64 + 64) + 64 * 64 + 64 + 8 * 64 + 8 == 21512
    assert G.n_weights(**SMALL) == (2 * 8 * 2 + 8) + (2 * 8 * 8 + 8) + 64 + 8 + 32 + 4


def test_permutation_invariance():
    w = _weights(3, **SMALL)
    n, edges = 9, I.erdos_renyi(9, 0.4, 11)
    perm = np.random.default_rng(0).permutation(n)
    edges_p = [(int(perm[a]), int(perm[b])) for a, b in edges]
    y0 = G.forward(w, *I.pack_graphs([(n, edges)]), **SMALL)
    y1 = G.forward(w, *I.pack_graphs([(n, edges_p)]), **SMALL)
    assert np.allclose(y0, y1, atol=1e-13, rtol=0)


def _mlp(P, h, layers):
    for l in range(layers):
        h = np.maximum((P[f"Ws{l}"] + P[f"Wn{l}"]) @ h + P[f"bl{l}"], 0.0)
    return P["W2"] @ np.maximum(P["W1"] @ h + P["b1"], 0.0) + P["b2"]


def test_regular_graph_reduces_to_mlp():
    # every node of a d-regular graph has the same features, so the mean over
    # neighbours equals the node's own embedding at every layer
    w = _weights(5, **SMALL)
    P = G.unpack(w, **SMALL)
    for d, n in ((3, 10), (4, 9), (2, 7)):
        edges = I.random_regular_graph(n, d, 7)
        y = G.forward(w, *I.pack_graphs([(n, edges)]), **SMALL)[0]
        assert np.allclose(y, _mlp(P, np.array([1.0, d / 3.0]), SMALL["layers"]), atol=1e-13)


def test_edgeless_and_empty_graphs():
    w = _weights(6, **SMALL)
    P = G.unpack(w, **SMALL)
    y = G.forward(w, *I.pack_graphs([(5, []), (0, [])]), **SMALL)
    h = np.array([1.0, 0.0])
    for l in range(SMALL["layers"]):
        h = np.maximum(P[f"Ws{l}"] @ h + P[f"bl{l}"], 0.0)  # no neighbours: a = 0
    want0 = P["W2"] @ np.maximum(P["W1"] @ h + P["b1"], 0.0) + P["b2"]
    want1 = P["W2"] @ np.maximum(P["b1"], 0.0) + P["b2"]  # empty graph: r = 0
    assert np.allclose(y[0], want0, atol=1e-13) and np.allclose(y[1], want1, atol=1e-13)


def test_backward_matches_finite_differences():
    w = _weights(8, **SMALL)
    graphs = [(7, I.erdos_renyi(7, 0.5, 1)), (6, I.random_regular_graph(6, 3, 2)), (4, [(0, 1), (1, 2)])]
    batch = I.pack_graphs(graphs)
    dy = np.random.default_rng(4).normal(size=(len(graphs), SMALL["out_dim"]))
    g = G.backward(w, *batch, dy, **SMALL)
    h = 1e-6
    fd = np.zeros_like(w)
    for i in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd[i] = (np.sum(dy * G.forward(wp, *batch, **SMALL)) - np.sum(dy * G.forward(wm, *batch, **SMALL))) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_mse_gradient():
    rng = np.random.default_rng(2)
    y, t = rng.normal(size=(3, 4)), rng.normal(size=(3, 4))
    loss, dy = G.mse(y, t)
    assert loss == pytest.approx(np.sum((y - t) ** 2) / 12)
    e = np.zeros_like(y)
    e[1, 2] = 1e-6
    assert dy[1, 2] == pytest.approx((G.mse(y + e, t)[0] - G.mse(y - e, t)[0]) / 2e-6, rel=1e-7)


def test_adam_first_steps():
    # step 1: bias-corrected m = g and v = g^2, so the update is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    w1, m, v = G.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.1)
    assert np.allclose(w1, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-15, atol=0)
    # two steps with g = +1 then -1, worked by hand:
    # m2 = -0.01, mhat2 = -0.01 / 0.19; v2 = 0.001999, vhat2 = 1
    w, m, v = G.adam(0.0, 0.0, 0.0, 1.0, 1, 0.1)
    w, m, v = G.adam(w, m, v, -1.0, 2, 0.1)
    assert float(w) == pytest.approx(-0.1 / (1 + 1e-8) + 0.1 * (0.01 / 0.19) / (1 + 1e-8), abs=1e-15)
