"""Multi-GPU host logic: instance partitioning across ranks, and the planner
for one state sharded across ranks (global qubits and swap schedule).

Partitioning (the batch dimension of the gradient operator, §4.1): independent
instances are dealt to ranks by a cost estimate (2^n amplitudes times gates:
one streaming sweep per gate of a 2^n state), largest first onto the least
loaded rank, so every rank evaluates its share with no collective on the data
path and one gather of the results at the end.

Sharding one state: with 2^g ranks, the top g physical qubit positions index
the rank and the low n - g are local to each rank's shard.  A gate whose
targets are all local runs on every shard (a control on a global position
becomes a rank predicate); a gate with a global target is preceded by a swap
of that global position with a local one, an exchange of half of every
shard between rank pairs.  ``plan_global_swaps`` chooses the swaps (the local
position evicted is the one whose qubit is next needed as a target furthest
in the future) and returns the schedule; energies and gradients then take one
FP64 all-reduce of per-rank partial sums.  Neither path has been run on more
than one GPU: both are tested on the CPU (gloo ranks, simulated shards).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Sequence, Tuple

import numpy as np


# ----------------------------------------------------------------------------- instance partition

def instance_cost(n_qubits: int, n_gates: int) -> float:
    """Work estimate of one evaluation: 2^n amplitudes swept once per gate."""
    return float(2 ** n_qubits) * float(max(n_gates, 1))


def partition_by_cost(costs: Sequence[float], world_size: int) -> List[List[int]]:
    """Longest-processing-time assignment: instances by decreasing cost (ties by
    index), each onto the rank with the smallest load so far (ties: lowest
    rank).  Deterministic; every rank's list is in increasing index order."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world_size
    parts: List[List[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def evaluate_partitioned(n_inst: int, costs: Sequence[float], evaluate: Callable[[List[int]], Tuple],
                         rank: int, world_size: int):
    """Evaluate this rank's share and gather every instance's results on all
    ranks (one all_gather_object; with world_size 1 no collective).

    evaluate(indices) -> (energies[len], grads: list of arrays) for those
    instances.  Returns (energies[n_inst], grads[n_inst])."""
    parts = partition_by_cost(costs, world_size)
    mine = parts[rank]
    e, g = evaluate(mine) if mine else (np.zeros(0), [])
    local = (mine, [float(v) for v in e], [np.asarray(x, dtype=np.float64) for x in g])
    if world_size > 1:
        import torch.distributed as dist
        allr = [None] * world_size
        dist.all_gather_object(allr, local)
    else:
        allr = [local]
    energies = np.zeros(n_inst)
    grads: List[np.ndarray] = [np.zeros(0)] * n_inst
    seen = np.zeros(n_inst, dtype=bool)
    for idx, es, gs in allr:
        for k, i in enumerate(idx):
            energies[i] = es[k]
            grads[i] = gs[k]
            seen[i] = True
    if not seen.all():
        raise RuntimeError("an instance was not evaluated by any rank")
    return energies, grads


# ----------------------------------------------------------------------------- sharded state planner

@dataclass
class ShardStep:
    kind: str                 # "gates": run gates[begin:end] on every shard; "swap": exchange positions
    begin: int = 0
    end: int = 0
    glob: int = -1            # swap: the global position (n - g .. n - 1)
    loc: int = -1             # swap: the local position (0 .. n - g - 1)


def plan_global_swaps(n: int, g: int, targets: Sequence[Sequence[int]]) -> Tuple[List[ShardStep], List[int]]:
    """Schedule for gates with the given target qubits on an n-qubit state
    sharded over 2^g ranks.  Physical positions n-g..n-1 are global.  Starts
    from the identity layout (qubit q at position q).

    Returns (steps, final layout): layout[q] = physical position of qubit q.
    Every gate's targets sit at local positions when its "gates" step runs;
    each "swap" exchanges the qubits at one global and one local position."""
    if not 0 <= g < n:
        raise ValueError("need 0 <= g < n")
    nl = n - g
    pos = list(range(n))            # qubit -> position
    at = list(range(n))             # position -> qubit
    steps: List[ShardStep] = []
    seg = 0

    def next_use(q: int, after: int) -> int:
        for k in range(after, len(targets)):
            if q in targets[k]:
                return k
        return len(targets) + 1

    for k, ts in enumerate(targets):
        if len(set(ts)) > nl:
            raise ValueError("a gate has more targets than local positions")
        need = [q for q in ts if pos[q] >= nl]
        if not need:
            continue
        if k > seg:
            steps.append(ShardStep("gates", seg, k))
        seg = k
        for q in need:
            # evict the local qubit (not a target of this gate) used furthest in the future
            cands = [p for p in range(nl) if at[p] not in ts]
            victim = max(cands, key=lambda p: (next_use(at[p], k), -p))
            gp = pos[q]
            qv = at[victim]
            steps.append(ShardStep("swap", glob=gp, loc=victim))
            pos[q], pos[qv] = victim, gp
            at[victim], at[gp] = q, qv
    if seg < len(targets):
        steps.append(ShardStep("gates", seg, len(targets)))
    return steps, pos


def swap_exchange_pairs(n: int, g: int, glob: int, loc: int) -> List[Tuple[int, int]]:
    """Rank pairs of one swap: the ranks differing in the global bit exchange
    the halves of their shards that differ in the local bit (rank r with bit
    b = 0 sends its local-bit-1 half to rank r | 2^b, which sends back its
    local-bit-0 half)."""
    b = glob - (n - g)
    return [(r, r | (1 << b)) for r in range(1 << g) if not (r >> b) & 1]
