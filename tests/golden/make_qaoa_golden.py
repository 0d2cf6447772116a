"""Writes tests/golden/qaoa24_p8.json with the FP64 oracle (and nothing else).

Workload: the 30-qubit QAOA benchmark recipe at 24 nodes -- a seeded random
3-regular graph (pairing model, seed 3), p = 8, RZZ(gamma_l) on every edge then
RX(beta_l) on every qubit (gamma_scale 0.5), 16 angles U[0, pi] (seed 3:
gamma_1..8 then beta_1..8), start |+>^24.  Run:  python tests/golden/make_qaoa_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import qsim_oracle as O  # noqa: E402
from paper_2406_17248_gb300 import inputs as I  # noqa: E402


def main(n=24, p=8, seed=3):
    edges = I.random_regular_graph(n, 3, seed)
    angles = I.uniform_params(2 * p, seed, 0.0, 3.141592653589793)
    t = time.time()
    E, dg, db = O.qaoa_expectation_with_grad(n, edges, angles[:p], angles[p:], 0.5)
    out = {
        "generator": "tests/golden/make_qaoa_golden.py (FP64 oracle)",
        "n": n, "p": p, "seed": seed, "gamma_scale": 0.5,
        "edges": [list(e) for e in edges],
        "gamma": list(angles[:p]), "beta": list(angles[p:]),
        "energy": E, "dgamma": list(dg), "dbeta": list(db),
        "oracle_seconds": time.time() - t,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"qaoa{n}_p{p}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, E, out["oracle_seconds"])


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:]))
