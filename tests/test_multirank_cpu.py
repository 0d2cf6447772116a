"""The N > 1 path of bench.py on the CPU (gloo, world size 2): the max-over-ranks
timing helper and barrier, and a two-rank launch of the reference arm under
torch.distributed.run in which rank 0 alone prints one JSON line.  The GPU path
runs one independent replica per rank (no collective on the data path), so the
cross-rank logic exercised here is all there is."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    m = bench.reduce_max(1.5 + rank, world)
    bench.barrier(world)
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}"), "w") as f:
        f.write(repr(m))


def test_reduce_max_and_barrier_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    assert [float((tmp_path / f"r{r}").read_text()) for r in range(2)] == [2.5, 2.5]


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--ref-qubits", "8"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


# ----------------------------------------------------------------------------- instance partition

def _small_instances():
    from paper_2406_17248_gb300 import inputs as I
    return I.batched_vqe(12, seed=9, n_range=(4, 7), depth_range=(1, 3))


def _oracle_eval(instances, idx):
    from oracle import qsim_oracle as O
    es, gs = [], []
    for i in idx:
        it = instances[i]
        n = it.circuit.n_qubits
        E, g = O.adjoint_gradient(it.circuit, it.ham, it.params, O.zero_state(n))
        es.append(E)
        gs.append(g)
    return es, gs


def test_partition_by_cost_is_a_balanced_cover():
    from paper_2406_17248_gb300 import distributed as D
    from paper_2406_17248_gb300 import inputs as I
    inst = I.batched_vqe(200, seed=4)
    costs = [D.instance_cost(it.circuit.n_qubits, len(it.circuit.gates)) for it in inst]
    for ws in (1, 2, 3, 8):
        parts = D.partition_by_cost(costs, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(inst)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # list scheduling: the largest load is within one instance of the mean
        assert max(loads) <= sum(costs) / ws + max(costs)
        assert parts == D.partition_by_cost(costs, ws)


def _partition_rank_main(rank, world, port, out):
    import pickle
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2406_17248_gb300 import distributed as D
    inst = _small_instances()
    costs = [D.instance_cost(it.circuit.n_qubits, len(it.circuit.gates)) for it in inst]
    dist.init_process_group("gloo", rank=rank, world_size=world)
    e, g = D.evaluate_partitioned(len(inst), costs, lambda idx: _oracle_eval(inst, idx), rank, world)
    dist.destroy_process_group()
    with open(os.path.join(out, f"p{rank}"), "wb") as f:
        pickle.dump((e, g, D.partition_by_cost(costs, world)[rank]), f)


def test_partitioned_batch_over_two_gloo_ranks_matches_one_rank(tmp_path):
    """Each rank evaluates its cost-balanced share (here with the FP64 oracle);
    one gather gives every rank all energies and gradients, identical to a
    single-rank evaluation."""
    import pickle
    import numpy as np
    import torch.multiprocessing as mp
    from paper_2406_17248_gb300 import distributed as D
    port = _free_port()
    mp.start_processes(_partition_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    inst = _small_instances()
    costs = [D.instance_cost(it.circuit.n_qubits, len(it.circuit.gates)) for it in inst]
    e1, g1 = D.evaluate_partitioned(len(inst), costs, lambda idx: _oracle_eval(inst, idx), 0, 1)
    shares = []
    for r in range(2):
        e, g, mine = pickle.load(open(tmp_path / f"p{r}", "rb"))
        shares.append(mine)
        assert np.array_equal(e, e1)
        assert all(np.array_equal(a, b) for a, b in zip(g, g1))
    assert sorted(shares[0] + shares[1]) == list(range(len(inst))) and shares[0] and shares[1]


# ----------------------------------------------------------------------------- sharded state planner

def _simulate_shards(circ, params, psi0, g):
    """Run a circuit on 2^g simulated shards following plan_global_swaps: gates
    on local positions per shard (controls at global positions as a rank
    predicate), swaps as exchanges of half-shards between rank pairs."""
    import numpy as np
    from oracle import qsim_oracle as O
    from paper_2406_17248_gb300 import distributed as D
    n = circ.n_qubits
    nl = n - g
    steps, layout = D.plan_global_swaps(n, g, [tuple(gt.targets) for gt in circ.gates])
    shards = [psi0.reshape(1 << g, 1 << nl)[r].copy() for r in range(1 << g)]  # identity layout at the start
    pos = list(range(n))
    for st in steps:
        if st.kind == "swap":
            b = st.glob - nl
            for r0, r1 in D.swap_exchange_pairs(n, g, st.glob, st.loc):
                assert (r0 ^ r1) == 1 << b
                a, c = shards[r0].reshape(-1, 2, 1 << st.loc), shards[r1].reshape(-1, 2, 1 << st.loc)
                tmp = a[:, 1, :].copy()
                a[:, 1, :] = c[:, 0, :]
                c[:, 0, :] = tmp
            qa = pos.index(st.glob)
            qb = pos.index(st.loc)
            pos[qa], pos[qb] = st.loc, st.glob
            continue
        for k in range(st.begin, st.end):
            gt = circ.gates[k]
            U = O.gate_unitary(gt, params)
            tl = [pos[q] for q in gt.targets]
            assert all(p < nl for p in tl), "a target at a global position"
            cl = [pos[q] for q in gt.ctrls if pos[q] < nl]
            cg = [pos[q] - nl for q in gt.ctrls if pos[q] >= nl]
            for r in range(1 << g):
                if all((r >> b) & 1 for b in cg):
                    shards[r] = O.apply_gate(shards[r], nl, U, tl, cl)
    assert pos == layout
    phys = np.concatenate(shards)
    x = np.arange(1 << n)
    p = np.zeros(1 << n, dtype=np.int64)
    for q in range(n):
        p |= ((x >> q) & 1) << pos[q]
    return phys[p], phys, pos


@pytest.mark.parametrize("n,g,seed", [(6, 1, 1), (8, 2, 2), (9, 3, 3)])
def test_sharded_state_plan_matches_the_oracle(n, g, seed):
    import numpy as np
    from oracle import qsim_oracle as O
    from paper_2406_17248_gb300 import inputs as I
    circ = I.random_mixed_circuit(n, 80, seed=seed, max_ctrls=2)
    params = I.uniform_params(circ.n_params, seed)
    psi0 = I.random_state(n, seed)
    from paper_2406_17248_gb300 import distributed as D
    steps, _ = D.plan_global_swaps(n, g, [tuple(gt.targets) for gt in circ.gates])
    assert sum(s.kind == "swap" for s in steps) >= 3  # the circuit does reach the global positions
    got, phys, pos = _simulate_shards(circ, params, psi0, g)
    want = O.evolve(circ, params, psi0)
    assert np.abs(got - want).max() < 1e-12
    # a Z-string energy: per-rank partial sums reduced once (the all-reduce)
    ham = I.pauli_sum_from_strings(n, [(0.7, "Z0 Z1"), (-0.3, f"Z{n - 1}"), (0.5, f"Z2 Z{n - 2}")])
    nl = n - g
    partial = []
    for r in range(1 << g):
        sh = phys[r << nl:(r + 1) << nl]
        l = np.arange(1 << nl)
        e = 0.0
        for cf, zm in zip(ham.coef, ham.zmask):
            par = np.zeros(1 << nl, dtype=np.int64)
            for q in range(n):
                if (int(zm) >> q) & 1:
                    pq = pos[q]
                    par ^= ((l >> pq) & 1) if pq < nl else ((r >> (pq - nl)) & 1)
            e += float(cf) * float(np.sum((1 - 2 * par) * np.abs(sh) ** 2))
        partial.append(e)
    assert abs(sum(partial) - O.expectation(want, ham)) < 1e-12


def test_swap_planner_keeps_targets_local_and_swaps_only_when_needed():
    from paper_2406_17248_gb300 import distributed as D
    n, g = 10, 3
    # gates on local qubits only: no swap
    steps, layout = D.plan_global_swaps(n, g, [(0,), (3, 5), (6,)])
    assert [s.kind for s in steps] == ["gates"] and layout == list(range(n))
    # one gate on a global qubit: exactly one swap, the evicted local qubit is one never used again
    steps, layout = D.plan_global_swaps(n, g, [(0,), (8,), (0,)])
    sw = [s for s in steps if s.kind == "swap"]
    assert len(sw) == 1 and sw[0].glob == 8 and sw[0].loc != 0 and layout[8] < n - g
