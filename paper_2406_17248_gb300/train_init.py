"""Train and evaluate the learned QAOA initialiser end to end on one GPU.

  python -m paper_2406_17248_gb300.train_init --train 2048 --test 256 --out result.json

1. labels: seeded random graphs (half 3-regular, half Erdos-Renyi G(n, 0.3)),
   QAOA angles optimised by the batched simulator (Adam from the linear ramp
   and from random starts, best kept, canonicalised);
2. training: the graph network regresses the labels (MSE, Adam), all on the
   device;
3. evaluation on held-out graphs: Adam from the network's prediction and from
   the linear ramp, steps until the approximation ratio reaches the target;
4. timing of one forward and one backward launch of the network.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--train-n", type=int, nargs=2, default=(10, 13))
    ap.add_argument("--restarts", type=int, default=4)
    ap.add_argument("--label-steps", type=int, default=200)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--test-n", type=int, nargs=2, default=(16, 18))
    ap.add_argument("--eval-steps", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--angle-lr", type=float, default=0.05)
    ap.add_argument("--target", type=float, default=0.9)
    ap.add_argument("--delta", type=float, default=0.75)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)

    import torch

    from . import inputs as I
    from . import qsim as Q
    from .qaoa_init import Initialiser, linear_ramp, optimised_angles, steps_to_ratio

    Q.lib()
    res = {"p": a.p, "train": a.train, "train_n": list(a.train_n), "test": a.test, "test_n": list(a.test_n),
           "target_ratio": a.target}
    train = I.graph_set(a.train, a.seed, tuple(a.train_n))
    test = I.graph_set(a.test, a.seed + 1000, tuple(a.test_n))

    t0 = time.perf_counter()
    labels, best_e = optimised_angles(train, a.p, restarts=a.restarts, steps=a.label_steps, lr=a.angle_lr,
                                      seed=a.seed, delta=a.delta)
    res["label_seconds"] = time.perf_counter() - t0
    res["label_evals"] = a.train * (a.restarts + 1) * (a.label_steps + 1)

    init = Initialiser(p=a.p, seed=a.seed)
    t0 = time.perf_counter()
    losses = init.fit(train, labels, epochs=a.epochs, batch_size=a.batch, lr=a.lr, seed=a.seed)
    res["train_seconds"] = time.perf_counter() - t0
    res["loss_first_last"] = [float(losses[0]), float(losses[-1])]

    # network launch timing on one full batch of test graphs
    gb = Q.Graphs.from_graphs(test[: a.batch])
    y = torch.zeros(gb.n_graphs, 2 * a.p, dtype=torch.float32, device="cuda")
    dy = torch.randn_like(y)
    grad = torch.zeros(init.net.n_weights, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(3):
        init.net.forward(gb, y)
        init.net.backward(gb, dy, grad)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    reps = 20
    ev[0].record(st)
    for _ in range(reps):
        init.net.forward(gb, y)
    ev[1].record(st)
    for _ in range(reps):
        init.net.backward(gb, dy, grad)
    ev[2].record(st)
    torch.cuda.synchronize()
    res["gnn_batch_graphs"] = gb.n_graphs
    res["gnn_forward_us"] = 1e3 * ev[0].elapsed_time(ev[1]) / reps
    res["gnn_backward_us"] = 1e3 * ev[1].elapsed_time(ev[2]) / reps

    pred = init.predict(test)
    ramp = np.tile(linear_ramp(a.p, a.delta), (len(test), 1))
    for name, start in (("learned", pred), ("ramp", ramp)):
        first, ratio, dt = steps_to_ratio(test, start, a.p, steps=a.eval_steps, lr=a.angle_lr, target=a.target)
        hit = first >= 0
        res[name] = {
            "fraction_reaching_target": float(hit.mean()),
            "mean_steps_when_reached": float(first[hit].mean()) if hit.any() else None,
            "median_steps_when_reached": float(np.median(first[hit])) if hit.any() else None,
            "ratio_at_step0_mean": float(ratio[0].mean()),
            "ratio_final_mean": float(ratio[-1].mean()),
            "seconds_all_graphs": dt,
            "seconds_per_step": dt / (a.eval_steps + 1),
        }
    line = json.dumps(res)
    print(line, flush=True)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
