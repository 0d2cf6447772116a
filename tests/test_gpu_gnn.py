"""GPU parity of the learned-initialiser kernels against the FP64 oracle:
bfloat16 rounding (bit-exact), forward and backward of the graph network, MSE,
Adam (float32 with bf16 shadow, and float64), the batched angle optimiser, the
device MaxCut, and a training run that must fit its targets."""
import math

import numpy as np
import pytest

from oracle import gnn_oracle as G
from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def Q():
    from paper_2406_17248_gb300 import qsim
    qsim.lib()
    return qsim


def _bf16_bits_to_f64(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _random_weights(seed, **dims):
    lay = [(k, r, c) for _, k, r, c in G.layout(**dims)]
    w = I.gnn_init_weights(lay, seed)
    rng = np.random.default_rng(seed + 100)
    o = 0
    for _, k, r, c in G.layout(**dims):
        if k == "b":
            w[o:o + r] = rng.uniform(-0.2, 0.2, size=r)
        o += r * c
    return w.astype(np.float32)


def _graph_mix(seed):
    gs = I.graph_set(20, seed, (4, 26))
    gs += [(0, []), (5, []), (1, []), (2, [(0, 1)]), (64, I.random_regular_graph(64, 3, seed)),
           (64, I.erdos_renyi(64, 0.3, seed)), (26, I.erdos_renyi(26, 0.9, seed))]
    return gs


def _pick_inputs(dims, margin=1e-5):
    """Weights and graphs whose ReLU pre-activations all stay `margin` away from
    zero (so float32 and float64 take the same derivative branch)."""
    for seed in range(50):
        w = _random_weights(seed, **dims)
        batch = I.pack_graphs(_graph_mix(seed))
        if G.min_abs_preactivation(G.bf16_round(w), *batch, **dims) > margin:
            return w, batch
    raise AssertionError("no seed with a ReLU margin")


@pytest.mark.parametrize("dims", [dict(hidden=64, layers=3, out_dim=8), dict(hidden=16, layers=2, out_dim=6)])
def test_gnn_forward_backward_parity(Q, dims):
    w, batch = _pick_inputs(dims)
    net = Q.GNN(dims["hidden"], dims["layers"], dims["out_dim"])
    net.set_weights(w)
    w_back, wb = net.get_weights()
    assert np.array_equal(w_back, w)
    wb64 = _bf16_bits_to_f64(wb)
    assert np.array_equal(wb64, G.bf16_round(w))  # round to nearest even, bit for bit
    graphs = Q.Graphs(*batch)
    nG = graphs.n_graphs
    y = torch.zeros(nG, dims["out_dim"], dtype=torch.float32, device="cuda")
    net.forward(graphs, y)
    y_or = G.forward(wb64, *batch, **dims)
    y_gpu = y.cpu().numpy().astype(np.float64)
    scale = max(1.0, np.max(np.abs(y_or)))
    assert np.max(np.abs(y_gpu - y_or)) <= 1e-4 * scale
    dy = np.random.default_rng(1).normal(size=y_or.shape)
    grad = torch.zeros(net.n_weights, dtype=torch.float32, device="cuda")
    net.backward(graphs, torch.as_tensor(dy, dtype=torch.float32).cuda(), grad)
    g_or = G.backward(wb64, *batch, dy.astype(np.float32).astype(np.float64), **dims)
    g_gpu = grad.cpu().numpy().astype(np.float64)
    gscale = max(1.0, np.max(np.abs(g_or)))
    assert np.max(np.abs(g_gpu - g_or)) <= 1e-4 * gscale
    # bitwise reproducible
    grad2 = torch.zeros_like(grad)
    net.backward(graphs, torch.as_tensor(dy, dtype=torch.float32).cuda(), grad2)
    assert torch.equal(grad, grad2)


def test_gnn_empty_batch_and_single_graph(Q):
    net = Q.GNN(8, 1, 2)
    net.set_weights(_random_weights(3, hidden=8, layers=1, out_dim=2))
    g0 = Q.Graphs(np.array([0]), np.array([0]), np.array([]))
    grad = torch.full((net.n_weights,), 7.0, dtype=torch.float32, device="cuda")
    net.forward(g0, torch.zeros(1, 2, device="cuda"))
    net.backward(g0, torch.zeros(1, 2, device="cuda"), grad)
    assert torch.count_nonzero(grad).item() == 0


def test_mse_and_adam_parity(Q):
    rng = np.random.default_rng(5)
    y, t = rng.normal(size=(37, 8)).astype(np.float32), rng.normal(size=(37, 8)).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    dy = torch.zeros(37, 8, device="cuda")
    Q.mse(torch.as_tensor(y).cuda(), torch.as_tensor(t).cuda(), loss, dy)
    l_or, dy_or = G.mse(y.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - l_or) <= 3e-5 * l_or
    assert np.max(np.abs(dy.cpu().numpy() - dy_or)) <= 1e-6 * np.max(np.abs(dy_or))
    # float32 Adam with bf16 shadow, three steps
    dims = dict(hidden=8, layers=1, out_dim=2)
    net = Q.GNN(8, 1, 2)
    w0 = _random_weights(9, **dims)
    net.set_weights(w0)
    wo, m, v = w0.astype(np.float64), np.zeros(w0.size), np.zeros(w0.size)
    for t_ in range(1, 4):
        g = rng.normal(size=w0.size).astype(np.float32)
        net.adam_step(torch.as_tensor(g).cuda(), 1e-2)
        wo, m, v = G.adam(wo, m, v, g.astype(np.float64), t_, 1e-2)
    w_gpu, wb = net.get_weights()
    assert np.max(np.abs(w_gpu - wo)) <= 1e-6 * max(1.0, np.max(np.abs(wo)))
    assert np.array_equal(_bf16_bits_to_f64(wb), G.bf16_round(w_gpu))
    # float64 Adam (maximize flips the gradient)
    n = 100
    w = torch.as_tensor(rng.normal(size=n)).cuda()
    mm, vv = torch.zeros(n, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda")
    wo, m, v = w.cpu().numpy(), np.zeros(n), np.zeros(n)
    for t_ in range(1, 6):
        g = rng.normal(size=n)
        Q.adam_f64(w, mm, vv, torch.as_tensor(g).cuda(), t_, 0.05, maximize=(t_ == 3))
        wo, m, v = G.adam(wo, m, v, -g if t_ == 3 else g, t_, 0.05)
    assert np.max(np.abs(w.cpu().numpy() - wo)) <= 1e-13


def test_max_cut_matches_brute_force(Q):
    from paper_2406_17248_gb300.qaoa_init import max_cuts
    gs = I.graph_set(6, 2, (6, 14)) + [(5, I.complete_graph(5)), (4, []), (3, [(0, 1), (1, 2)])]
    want = [O.maxcut_brute_force(n, e) for n, e in gs]
    assert max_cuts(gs).astype(int).tolist() == want


def test_angle_optimiser_matches_oracle_trajectory(Q):
    # complex128 batch: gradients to ~1e-12, so Adam trajectories agree closely
    from paper_2406_17248_gb300.qaoa_init import AngleOptimiser, linear_ramp
    p = 2
    gs = I.graph_set(3, 4, (6, 9))
    init = np.stack([linear_ramp(p, 0.6 + 0.1 * i) for i in range(len(gs))])
    opt = AngleOptimiser(gs, p, dtype=Q.C128)
    final, hist, _ = opt.run(init, 6, lr=0.05)
    for i, (n, e) in enumerate(gs):
        a, m, v = init[i].copy(), np.zeros(2 * p), np.zeros(2 * p)
        for t_ in range(1, 7):
            E, dg, db = O.qaoa_expectation_with_grad(n, e, a[:p], a[p:], gamma_scale=0.5)
            assert abs(hist[t_ - 1, i] - E) <= 1e-10 * max(1, len(e))
            a, m, v = G.adam(a, m, v, np.concatenate([dg, db]), t_, 0.05)
        assert np.max(np.abs(final[i] - a)) <= 1e-9
        assert abs(hist[-1, i] - O.qaoa_expectation_with_grad(n, e, a[:p], a[p:], gamma_scale=0.5)[0]) <= 1e-9


def test_training_fits_targets(Q):
    # targets that depend on the graph (mean degree): the network must fit them
    from paper_2406_17248_gb300.qaoa_init import Initialiser
    gs = I.graph_set(96, 8, (6, 14))
    md = np.array([2.0 * len(e) / n for n, e in gs])
    targets = np.stack([0.3 + 0.1 * md, -0.5 + 0.05 * md, 0.2 * np.ones_like(md), -0.1 * md], axis=1)
    init = Initialiser(p=2, hidden=32, layers=2, seed=1)
    losses = init.fit(gs, targets, epochs=150, batch_size=32, lr=3e-3, seed=2)
    assert losses[-1] < 0.02 * losses[0]
    pred = init.predict(gs)
    assert np.sqrt(np.mean((pred - targets) ** 2)) < 0.05


def test_steps_to_ratio_engines_agree(Q):
    # the batched engine and the fused-pass QAOA engine run the same Adam
    # trajectories (complex64 both: agreement to float32 accuracy)
    from paper_2406_17248_gb300.qaoa_init import linear_ramp, steps_to_ratio
    p = 2
    gs = I.graph_set(4, 6, (8, 11))
    init = np.tile(linear_ramp(p), (len(gs), 1))
    f1, r1, _ = steps_to_ratio(gs, init, p, steps=5, lr=0.02, engine="batch")
    f2, r2, _ = steps_to_ratio(gs, init, p, steps=5, lr=0.02, engine="qaoa")
    assert np.max(np.abs(r1 - r2)) < 1e-4
    for i, (n, e) in enumerate(gs):
        E = O.qaoa_expectation_with_grad(n, e, init[i, :p], init[i, p:], gamma_scale=0.5)[0]
        assert abs(r2[0, i] - (len(e) - E) / 2 / O.maxcut_brute_force(n, e)) < 1e-5


def test_gnn_bench_batch_forward_and_sampled_backward(Q):
    """The benchmark batch (256 graphs of 26 nodes, hidden 64, 3 layers, seed 5)
    in the launch configuration bench.py times: the forward pass of every graph
    against the oracle; the backward pass on 24 sampled graphs whose ReLU inputs
    keep a margin from the kink."""
    from paper_2406_17248_gb300.qaoa_init import Initialiser
    graphs = I.graph_set(256, 5, (26, 26))
    init = Initialiser(p=4, seed=5)
    _, wb = init.net.get_weights()
    w64 = _bf16_bits_to_f64(wb)
    gb = Q.Graphs.from_graphs(graphs)
    y = torch.zeros(len(graphs), 8, dtype=torch.float32, device="cuda")
    init.net.forward(gb, y)
    y_or = G.forward(w64, *I.pack_graphs(graphs))
    assert np.max(np.abs(y.cpu().numpy() - y_or)) <= 1e-4 * max(1.0, np.max(np.abs(y_or)))
    sample = []
    for i in range(len(graphs)):
        if G.min_abs_preactivation(w64, *I.pack_graphs([graphs[i]])) > 1e-5:
            sample.append(graphs[i])
        if len(sample) == 24:
            break
    assert len(sample) == 24
    batch = I.pack_graphs(sample)
    dy = np.random.default_rng(3).normal(size=(len(sample), 8)).astype(np.float32)
    grad = torch.zeros(init.net.n_weights, dtype=torch.float32, device="cuda")
    init.net.backward(Q.Graphs(*batch), torch.as_tensor(dy).cuda(), grad)
    g_or = G.backward(w64, *batch, dy.astype(np.float64))
    assert np.max(np.abs(grad.cpu().numpy() - g_or)) <= 1e-4 * max(1.0, np.max(np.abs(g_or)))


def test_fused_train_step_equals_separate_calls(Q):
    """qs_gnn_train_step (two launches) gives the same weights bit for bit as
    forward + MSE + backward + Adam, and the loss to float32 rounding; the
    loss matches the oracle's MSE of the oracle forward pass."""
    dims = dict(hidden=64, layers=3, out_dim=8)
    w0 = _random_weights(4, **dims)
    graphs = I.graph_set(40, 12, (6, 26))
    targets = np.random.default_rng(2).normal(size=(len(graphs), 8)).astype(np.float32)
    gb = Q.Graphs.from_graphs(graphs)
    t = torch.as_tensor(targets).cuda()
    a, b = Q.GNN(64, 3, 8), Q.GNN(64, 3, 8)
    a.set_weights(w0)
    b.set_weights(w0)
    loss_a = torch.zeros(1, device="cuda")
    for _ in range(3):
        a.train_step(gb, t, 1e-3, loss_a)
    y = torch.zeros(len(graphs), 8, device="cuda")
    dy = torch.zeros_like(y)
    grad = torch.zeros(b.n_weights, device="cuda")
    loss_b = torch.zeros(1, device="cuda")
    for _ in range(3):
        b.forward(gb, y)
        Q.mse(y, t, loss_b, dy)
        b.backward(gb, dy, grad)
        b.adam_step(grad, 1e-3)
    wa, wba = a.get_weights()
    wb_, wbb = b.get_weights()
    assert np.array_equal(wa, wb_) and np.array_equal(wba, wbb)
    assert abs(loss_a.item() - loss_b.item()) <= 1e-5 * loss_b.item()
    # the loss of the last step was taken before its update: compare with the
    # oracle on the weights in force at that step (two steps applied)
    c = Q.GNN(64, 3, 8)
    c.set_weights(w0)
    for _ in range(2):
        c.train_step(gb, t, 1e-3)
    _, wbc = c.get_weights()
    y_or = G.forward(_bf16_bits_to_f64(wbc), *I.pack_graphs(graphs))
    l_or, _ = G.mse(y_or, targets.astype(np.float64))
    assert abs(loss_a.item() - l_or) <= 1e-4 * l_or


def test_training_state_checkpoint_and_resume(Q, tmp_path):
    """save() after three steps, then three more steps, equals load() into a fresh
    network followed by the same three steps, bit for bit (weights, bfloat16
    copy and Adam moments restored with the step count)."""
    dims = dict(hidden=64, layers=3, out_dim=8)
    w0 = _random_weights(5, **dims)
    graphs = I.graph_set(24, 13, (6, 26))
    targets = np.random.default_rng(3).normal(size=(len(graphs), 8)).astype(np.float32)
    gb = Q.Graphs.from_graphs(graphs)
    t = torch.as_tensor(targets).cuda()
    a = Q.GNN(64, 3, 8)
    a.set_weights(w0)
    for _ in range(3):
        a.train_step(gb, t, 1e-3)
    path = str(tmp_path / "gnn.npz")
    a.save(path)
    for _ in range(3):
        a.train_step(gb, t, 1e-3)
    b = Q.GNN(64, 3, 8).load(path)
    for _ in range(3):
        b.train_step(gb, t, 1e-3)
    wa, wba = a.get_weights()
    wb_, wbb = b.get_weights()
    assert np.array_equal(wa, wb_) and np.array_equal(wba, wbb)
    with pytest.raises(ValueError):
        Q.GNN(32, 3, 8).load(path)


def test_learned_initialiser_gains_over_linear_ramp(Q):
    """The whole learned part end to end at test size: labels optimised by the
    simulator (batched engine), the network trained by its own kernels, then on
    held-out larger graphs the network's angles start closer to the optimum than
    the plain linear-ramp initialisation (the fallback) and reach ratio 0.9 in
    fewer Adam steps, the simulator's energy deciding the ratio."""
    from paper_2406_17248_gb300.qaoa_init import Initialiser, linear_ramp, optimised_angles, steps_to_ratio
    p = 4
    train = I.graph_set(1024, 5, (10, 12))
    test = I.graph_set(48, 1005, (14, 16))
    labels, _ = optimised_angles(train, p, restarts=3, steps=120, lr=0.05, seed=5, delta=0.75)
    init = Initialiser(p=p, seed=5)
    losses = init.fit(train, labels, epochs=100, batch_size=256, lr=1e-3, seed=5)
    assert losses[-1] < 0.6 * losses[0]
    res = {}
    for name, start in (("learned", init.predict(test)), ("ramp", np.tile(linear_ramp(p, 0.75), (len(test), 1)))):
        first, ratio, _ = steps_to_ratio(test, start, p, steps=40, lr=0.05, target=0.9)
        res[name] = (float(ratio[0].mean()), first)
    assert res["learned"][0] > res["ramp"][0] + 0.02
    fl, fr = res["learned"][1], res["ramp"][1]
    both = (fl >= 0) & (fr >= 0)
    assert both.sum() >= 10
    assert np.median(fl[both]) < np.median(fr[both])
