"""Host-side pieces of the learned initialiser: the symmetry canonicalisation
(checked against oracle energies), the ramp, and the C-ABI's graph validation
(runs before any device work, so no GPU is needed)."""
import math

import numpy as np
import pytest

from oracle import gnn_oracle as G
from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I
from paper_2406_17248_gb300 import qsim as Q
from paper_2406_17248_gb300.qaoa_init import canonicalise, linear_ramp


def _energy(n, e, a, p):
    return O.qaoa_expectation_with_grad(n, e, a[:p], a[p:], gamma_scale=0.5)[0]


@pytest.mark.parametrize("seed", range(4))
def test_canonicalise_keeps_energy(seed):
    p = 3
    rng = np.random.default_rng(seed)
    n, e = I.graph_set(2, seed, (7, 9))[seed % 2]
    a = rng.uniform(-4, 4, size=2 * p)
    c = canonicalise(a, p)
    assert abs(_energy(n, e, a, p) - _energy(n, e, c, p)) < 1e-12
    assert np.all(c[:p] >= -math.pi) and np.all(c[:p] < math.pi) and c[0] >= 0
    assert np.all(c[p:] >= -math.pi / 2) and np.all(c[p:] < math.pi / 2)
    # every symmetry image has the same representative
    shift = np.concatenate([2 * math.pi * rng.integers(-2, 3, p), math.pi * rng.integers(-2, 3, p)])
    assert np.allclose(canonicalise(a + shift, p), c, atol=1e-12)
    assert np.allclose(canonicalise(-(a + shift), p), c, atol=1e-12)


def test_linear_ramp_closed_form_and_quality():
    a = linear_ramp(4, 0.75)
    assert np.allclose(a, [0.1875, 0.5625, 0.9375, 1.3125, -1.3125, -0.9375, -0.5625, -0.1875])
    # the ramp follows the adiabatic path towards low energy: well above the
    # random-assignment ratio of 1/2 on a 3-regular graph
    n, e = 12, I.random_regular_graph(12, 3, 1)
    ratio = (len(e) - _energy(n, e, a, 4)) / 2 / O.maxcut_brute_force(n, e)
    assert ratio > 0.8


def test_gnn_weight_count_matches_oracle():
    assert Q.gnn_n_weights(64, 3, 8) == G.n_weights() == 21512
    assert Q.gnn_n_weights(8, 2, 4) == G.n_weights(hidden=8, layers=2, out_dim=4)


@pytest.mark.parametrize("bad", ["too_many_nodes", "self_loop", "asymmetric", "repeat", "range"])
def test_graph_validation(bad):
    node_off, adj_off, adj = I.pack_graphs([(5, [(0, 1), (1, 2), (3, 4)])])
    if bad == "too_many_nodes":
        node_off, adj_off, adj = I.pack_graphs([(65, [(0, 1)])])
    elif bad == "self_loop":
        adj = adj.copy(); adj[0] = 0
    elif bad == "asymmetric":
        adj = adj.copy(); adj[0] = 2
    elif bad == "repeat":
        node_off, adj_off, adj = np.array([0, 2]), np.array([0, 2, 3]), np.array([1, 1, 0])
    elif bad == "range":
        adj = adj.copy(); adj[-1] = 7
    with pytest.raises(Q.QSimError) as ex:
        Q.Graphs(node_off, adj_off, adj)
    assert ex.value.status == 1


def test_density_matrix_channel_validation():
    """Channel arguments are checked on the host before any device work."""
    c = Q.DensityCircuit(3)
    c.add("H", (0,)).add_channel("depolarizing", 0, (0.2,))
    for kind, p, kraus in [("depolarizing", (1.5,), None), ("pauli", (0.5, 0.4, 0.3), None),
                           ("amplitude_damping", (-0.1,), None),
                           ("kraus", (), [np.eye(2), np.eye(2)])]:
        with pytest.raises(Q.QSimError) as ex:
            c.add_channel(kind, 1, p, kraus=kraus)
        assert ex.value.status == 1
    with pytest.raises(Q.QSimError):
        c.add_channel("depolarizing", 3, (0.1,))  # qubit beyond the system
