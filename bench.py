"""Benchmark: adjoint energy + gradient evaluations of 30-qubit complex64 QAOA.

Workload (the 30-qubit QAOA MaxCut configuration): a seeded random 3-regular
graph on 30 nodes (pairing model, seed 3, 45 edges), p = 8 layers of RZZ(gamma_l)
on every edge then RX(beta_l) on every qubit, 16 angles U[0, pi] (seed 3),
complex64 state from |+>^30 (8.6 GB, larger than L2, so no flush is needed).
One step = one call of qs_qaoa_expectation_with_grad: energy <C> and its 16
gradient entries by the adjoint method.

Run:  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
Prints one JSON line (rank 0).  With N > 1 (torchrun), every rank evaluates its
own independent angle vector (replicas: the evaluations share nothing) and the
value is the sum of evaluations over all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "30q c64 adjoint energy+grad evals/s; HBM GB/s vs peak; batched vs plain"
FALLBACK_HBM_GBS = 6800.0


def workload(n=30, p=8, seed=3):
    from paper_2406_17248_gb300 import inputs as I
    import numpy as np
    edges = I.random_regular_graph(n, 3, seed)
    angles = I.uniform_params(2 * p, seed, 0.0, float(np.pi))
    return edges, angles[:p], angles[p:]


def config(n, p, n_edges):
    return {"workload": f"QAOA MaxCut energy+adjoint gradient, {n} qubits, 3-regular graph (seed 3, {n_edges} edges), "
                        f"p={p}, complex64 from |+>^{n}",
            "n_qubits": n, "p": p, "edges": n_edges, "params": 2 * p, "state_dtype": "complex64",
            "l2": "state 2^30 x 8 B = 8.6 GB > L2; no flush needed", "parallelism": "replicas"}


# --------------------------------------------------------------------------- distributed helpers

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, ws: int) -> float:
    """Max of a float over ranks (identity for one rank)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- roofline inputs

def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    """Hash of the sources of the complex64 QAOA pass kernels (the counters in the
    committed ncu summary are valid only for this exact source)."""
    h = hashlib.sha256()
    for f in ("k_qaoa_x.cu", "qaoa_x.h", "qaoa_x_plan.cu"):
        with open(os.path.join(ROOT, "paper_2406_17248_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_launch(kind):
    """DRAM bytes per launch of a QAOA pass kernel kind from the committed ncu
    summary (a smaller capture scaled to 30 qubits), if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "qaoa_passes_qaoa30.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_full_launch\[%s\]:\s*([0-9.eE+]+)" % re.escape(kind), text)
    if not (m_hash and m_tr) or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_tr.group(1))


# --------------------------------------------------------------------------- CPU oracle

def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:  # Arm: /proc/cpuinfo has part numbers only; lscpu names the core
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=30).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(n_small, p, evals, threads, warmup=0):
    """Time the C FP64 oracle (one loop per gate, OpenMP over amplitudes) on the
    same recipe at n_small qubits in a child process without the GPU: (evals/s,
    seconds, threads used)."""
    code = (
        "import sys,time; sys.path.insert(0, %r)\n"
        "from oracle import qaoa_c\n"
        "from bench import workload\n"
        "e,g,b = workload(%d,%d)\n"
        "th = %d or qaoa_c.max_threads()\n"
        "for _ in range(%d): qaoa_c.evaluate(%d, e, g, b, 0.5, th)\n"
        "t=time.perf_counter()\n"
        "for _ in range(%d): qaoa_c.evaluate(%d, e, g, b, 0.5, th)\n"
        "print(time.perf_counter()-t, th)\n" % (ROOT, n_small, p, threads, warmup, n_small, evals, n_small))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    env.pop("OMP_NUM_THREADS", None)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr)
    sec, th = out.stdout.strip().splitlines()[-1].split()
    return evals / float(sec), float(sec), int(th)


def cpu_baseline_block(n, n_cpu, p):
    """The oracle measured at n_cpu qubits (not scaled to n): one evaluation on
    one thread, two on every host core."""
    r1, s1, _ = oracle_sample(n_cpu, p, 1, 1)
    ra, sa, tha = oracle_sample(n_cpu, p, 2, 0)
    return {"value": ra, "unit": "evals/s", "cores": tha, "kind": "oracle", "n_qubits": n_cpu,
            "sample": f"FP64 C oracle, the same recipe at {n_cpu} qubits (seeded 3-regular graph, p={p}), "
                      f"2 evaluations on {tha} threads ({sa:.1f} s); measured at {n_cpu} qubits, not scaled "
                      f"to the {n}-qubit workload",
            "single_thread": {"value": r1, "unit": "evals/s", "cores": 1, "seconds": s1},
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


# --------------------------------------------------------------------------- arms

def run_reference(args, ws, rank):
    """The oracle as it stands on the host cores: each step one evaluation of the
    recipe at --ref-qubits (24) qubits on every core, measured, not scaled."""
    if rank != 0:
        return
    n, p = args.n, args.p
    edges, _, _ = workload(n, p)
    ns = args.ref_qubits
    rate, sec, cores = oracle_sample(ns, p, args.steps, 0, warmup=args.warmup)
    line = {"metric": METRIC, "value": rate, "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(n, p, len(edges)),
            "impl": "reference",
            "cpu_baseline": {"value": rate, "unit": "evals/s", "cores": cores, "kind": "oracle", "n_qubits": ns,
                             "sample": f"{args.steps} FP64 C oracle evaluations of the recipe at {ns} qubits on "
                                       f"{cores} threads ({sec:.1f} s), after {args.warmup} warm-up; measured at "
                                       f"{ns} qubits, not scaled to the {n}-qubit workload",
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": rate, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim as Q

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    n, p = args.n, args.p
    edges, gam, bet = workload(n, p)
    if rank > 0:  # an independent evaluation per replica
        from paper_2406_17248_gb300 import inputs as I
        a = I.uniform_params(2 * p, 1000 + rank, 0.0, float(np.pi))
        gam, bet = a[:p], a[p:]
    q = Q.QAOA(n, edges, p, gamma_scale=0.5, dtype=Q.C64, tile_bits=args.tile_bits, low_bits=args.low_bits,
               checkpoint=args.checkpoint)
    info = q.info()
    psi, lam = Q.State(n, Q.C64), Q.State(n, Q.C64)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        q.expectation_with_grad(psi, lam, gam, bet)
    torch.cuda.synchronize()

    # ---- device-timed region: K evaluations, CUDA events on the launching stream
    clocks = ClockSampler(local)
    clocks.start()
    Q.trace_enable(True)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        E, dg, db = q.expectation_with_grad(psi, lam, gam, bet)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    Q.trace_enable(False)
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    k_ms, k_bytes, k_kind = Q.trace_read()
    ms_max = reduce_max(ms, ws)
    value = ws * args.steps / (ms_max / 1000.0)

    # ---- end to end through the public API with host inputs/outputs, host clock
    barrier(ws)
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for _ in range(args.steps):
        E2, dg2, db2 = q.expectation_with_grad(psi, lam, np.asarray(gam), np.asarray(bet))
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - h0, ws)
    n_coef = (2 * (len(edges) + 1) + 2) * p
    h2d = 2 * p * 8 + n_coef * 8
    d2h = (1 + 2 * p) * 8

    if rank != 0:
        return
    # roofline of the dominant kernel (the kernel with the most time in the step):
    # its algorithmic bytes per launch / its launch durations (CUDA events)
    peak, peak_kind = measured_peak_hbm()
    per_kind = {}
    for kd in sorted(set(int(x) for x in k_kind)):
        sel = k_kind == kd
        t = float(np.sum(k_ms[sel]))
        per_kind[Q.TRACE_KINDS[kd]] = {"launches_per_step": int(sel.sum()) // max(args.steps, 1),
                                       "ms_per_step": t / max(args.steps, 1),
                                       "GBps": float(np.sum(k_bytes[sel])) / (t / 1e3) / 1e9 if t > 0 else None,
                                       "bytes_per_launch": float(np.mean(k_bytes[sel]))}
    dom = max(per_kind, key=lambda k: per_kind[k]["ms_per_step"])
    achieved = per_kind[dom]["GBps"]
    all_ms = float(np.sum(k_ms))
    all_achieved = float(np.sum(k_bytes)) / (all_ms / 1000.0) / 1e9 if all_ms > 0 else None
    traffic = ncu_traffic_per_launch(dom)
    launches_per_step = len(k_ms) / max(args.steps, 1) + 2  # + slot reduction and output gather
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(n, p, len(edges)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs", "kernel": dom,
                     "bytes_per_launch": per_kind[dom]["bytes_per_launch"],
                     "all_passes_achieved": all_achieved,
                     "traced_share_of_step": all_ms / ms if ms > 0 else None,
                     "per_kernel": per_kind},
        "e2e": {"value": ws * args.steps / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk,
        "plan": info,
        "energy": E,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_block(n, args.cpu_qubits, p)
    if ws == 1 and not args.no_extras:
        # the rest of the headline: the single-gate sweep against the HBM roofline
        # and batched vs one-launch-per-circuit (untimed by the step clock above)
        del psi, lam, q
        torch.cuda.empty_cache()
        sw = measure_gate_sweep(Q, n, Q.C64, 3)
        line["gate_sweep"] = {k: sw[k] for k in ("n_qubits", "dtype", "GBps", "frac", "gates_per_s", "launches")}
        line["gate_sweep"]["per_kind_frac_median"] = {k: v["frac_median"] for k, v in sw["per_kind"].items()}
        line["random28"] = measure_random_c64(Q)
        line["random28"]["library_kernels"] = measure_random_c64(Q, fuse=3)
        line["batched_vs_plain"] = measure_batched_vs_plain(Q, args.instances, 3, args.plain_instances)
    print(json.dumps(line), flush=True)


def measure_batched_vs_plain(Q, instances, steps, plain_instances, warmup=3):
    """The batched-VQE recipe (n ~ U{10..20}, HEA depth ~ U{2..10}, TFIM, seed 4):
    one persistent launch per step (CUDA events) vs one launch sequence per
    circuit through the single-instance engine (host clock, synchronised)."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import inputs as I
    inst = I.batched_vqe(instances, seed=4)
    b = Q.Batch(inst, Q.C64)
    params = torch.tensor(np.concatenate([it.params for it in inst]), dtype=torch.float64, device="cuda")
    energies = torch.empty(len(inst), dtype=torch.float64, device="cuda")
    grads = torch.empty_like(params)
    for _ in range(warmup):
        b.expectation_with_grad_device(params, energies, grads)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        b.expectation_with_grad_device(params, energies, grads)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    batched = len(inst) / (ms / 1e3)
    plain_n = min(len(inst), plain_instances)
    circs = [Q.circuit_from(it.circuit).finalize(Q.C64) for it in inst[:plain_n]]
    hams = [Q.Hamiltonian(it.ham) for it in inst[:plain_n]]
    states = {}
    for it in inst[:plain_n]:
        n = it.circuit.n_qubits
        if n not in states:
            states[n] = (Q.State(n, Q.C64), Q.State(n, Q.C64))

    def plain_pass():
        for it, c, h in zip(inst[:plain_n], circs, hams):
            psi, lam = states[it.circuit.n_qubits]
            psi.set_basis(0)
            Q.expectation_with_grad(psi, lam, c, h, it.params)

    plain_pass()
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    plain_pass()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - h0
    plain = plain_n / plain_s
    e_b = energies.cpu().numpy()[:plain_n]
    psi, lam = states[inst[0].circuit.n_qubits]
    psi.set_basis(0)
    e0, _ = Q.expectation_with_grad(psi, lam, circs[0], hams[0], inst[0].params)
    return {"instances": len(inst), "batched": batched, "ms_per_step": ms, "steps": steps,
            "plain": plain, "plain_instances_timed": plain_n, "plain_seconds": plain_s,
            "speedup_vs_plain": batched / plain, "energy_check": abs(float(e_b[0]) - e0), "batch_info": b.info()}


def run_batch_workload(args):
    """2048 batched-VQE instances (n ~ U{10..20}, HEA depth ~ U{2..10}, TFIM, seed 4):
    one persistent launch per step vs one launch sequence per circuit."""
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    ws, rank, local = dist_setup()
    if ws > 1:
        return run_batch_partitioned(Q, args, ws, rank, local)
    r = measure_batched_vs_plain(Q, args.instances, args.steps, args.plain_instances, args.warmup)
    line = {"metric": "batched VQE energy+adjoint-grad instances/s (persistent launch vs one launch sequence per circuit)",
            "value": r["batched"], "unit": "instances/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{r['instances']} instances, n ~ U{{10..20}}, HEA depth ~ U{{2..10}}, TFIM "
                                   "J~N(1,0.2) h~U[0.5,1.5], complex64, seed 4", "instances": r["instances"]},
            "plain": {"value": r["plain"], "unit": "instances/s", "instances_timed": r["plain_instances_timed"],
                      "seconds": r["plain_seconds"]},
            "speedup_vs_plain": r["speedup_vs_plain"], "energy_check": r["energy_check"], "batch_info": r["batch_info"]}
    print(json.dumps(line), flush=True)


def run_batch_partitioned(Q, args, ws, rank, local):
    """The batch over N ranks (strong scaling: the instance set is fixed): each
    rank evaluates its cost-balanced share (2^n x gates, longest first) in its
    own persistent launch, with no collective on the data path; one gather of
    the energies at the end checks that every instance was evaluated."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2406_17248_gb300 import distributed as D
    from paper_2406_17248_gb300 import inputs as I
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    inst = I.batched_vqe(args.instances, seed=4)
    costs = [D.instance_cost(it.circuit.n_qubits, len(it.circuit.gates)) for it in inst]
    mine = D.partition_by_cost(costs, ws)[rank]
    sub = [inst[i] for i in mine]
    b = Q.Batch(sub, Q.C64)
    params = torch.tensor(np.concatenate([it.params for it in sub]), dtype=torch.float64, device="cuda")
    energies = torch.empty(len(sub), dtype=torch.float64, device="cuda")
    grads = torch.empty_like(params)
    for _ in range(args.warmup):
        b.expectation_with_grad_device(params, energies, grads)
    barrier(ws)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        b.expectation_with_grad_device(params, energies, grads)
    t1.record()
    torch.cuda.synchronize()
    barrier(ws)
    ms = reduce_max(t0.elapsed_time(t1) / args.steps, ws)
    allr = [None] * ws
    dist.all_gather_object(allr, (mine, energies.cpu().numpy().tolist()))
    if rank == 0:
        seen = sorted(i for idx, _ in allr for i in idx)
        assert seen == list(range(len(inst))), "an instance was not evaluated"
        line = {"metric": "batched VQE energy+adjoint-grad instances/s", "value": len(inst) / (ms / 1e3),
                "unit": "instances/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{len(inst)} instances, n ~ U{{10..20}}, HEA depth ~ U{{2..10}}, TFIM, "
                                       "complex64, seed 4; instances partitioned by 2^n x gates",
                           "instances": len(inst), "parallelism": f"instances over {ws} ranks"}}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def measure_random_c64(Q, n=28, G=500, reps=5, warmup=3, fuse=1):
    """The 28-qubit random circuit (500 gates over {H, RX, RY, RZ, CNOT, CZ},
    seed 2) on complex64 fused passes: gates/s and the passes' HBM roofline
    (algorithmic bytes of the traced passes / their CUDA-event time).  fuse = 1
    (the default): the passes compiled for the circuit; fuse = 3: the library's
    precompiled micro-op kernels."""
    import torch
    from paper_2406_17248_gb300 import inputs as I
    circ = I.random_circuit(n, G, seed=2)
    t_fin = time.perf_counter()
    c = Q.circuit_from(circ).finalize(Q.C64, fuse=fuse)
    t_fin = time.perf_counter() - t_fin
    s = Q.State(n, Q.C64)
    for _ in range(warmup):
        s.set_basis(0)
        c.apply(s)
    torch.cuda.synchronize()
    Q.trace_enable(True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        s.set_basis(0)
        c.apply(s)
    t1.record()
    torch.cuda.synchronize()
    Q.trace_enable(False)
    k_ms, k_by, k_kind = Q.trace_read()
    ms = t0.elapsed_time(t1) / reps
    peak, peak_kind = measured_peak_hbm()
    gbps = float(k_by.sum() / (k_ms.sum() / 1e3) / 1e9) if len(k_ms) else None
    micro = int((k_kind == 10).sum()) // reps
    gen = int((k_kind == 11).sum()) // reps
    del s
    torch.cuda.empty_cache()
    return {"n_qubits": n, "gates": G, "dtype": "c64", "fuse": fuse, "gates_per_s": G / (ms / 1e3), "ms": ms,
            "passes": c.info()["passes"], "micro_op_passes": micro, "generated_passes": gen,
            "finalize_s": t_fin, "GBps": gbps, "peak": peak,
            "frac": gbps / peak if gbps else None, "peak_source": f"{peak_kind} hbm_gbs",
            "note": "state reset to |0...0> each repetition (set_basis, inside the timed region)"}


def run_random_workload(args):
    """500-gate random circuit over {H, RX, RY, RZ, CNOT, CZ} on 28 qubits (seed 2),
    complex64 and complex128, fused tile passes vs one kernel per gate."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build, inputs as I
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    n, G = args.n, 500
    circ = I.random_circuit(n, G, seed=2)
    out = {}
    zsum = I.pauli_sum_from_strings(n, [(1.0, f"Z{q}") for q in range(n)])
    H = Q.Hamiltonian(zsum)
    for name, dt in (("c64", Q.C64), ("c128", Q.C128)):
        s = Q.State(n, dt)
        modes = (("fused", 1), ("library_kernels", 3), ("per_gate", -1)) if name == "c64" else (("fused", 1), ("per_gate", -1))
        for mode, fuse in modes:
            c = Q.circuit_from(circ).finalize(dt, fuse=fuse)
            s.set_basis(0)
            c.apply(s)
            torch.cuda.synchronize()
            Q.trace_enable(True)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = args.steps
            t0.record()
            for _ in range(reps):
                s.set_basis(0)
                c.apply(s)
            t1.record()
            torch.cuda.synchronize()
            Q.trace_enable(False)
            k_ms, k_by, _ = Q.trace_read()
            ms = t0.elapsed_time(t1) / reps
            amp = 8 if dt == Q.C64 else 16
            unfused = G * 2 * amp * (1 << n)
            out[f"{name}_{mode}"] = {"gates_per_s": G / (ms / 1e3), "ms": ms, "passes": c.info()["passes"],
                                     "effective_GBps": unfused / (ms / 1e3) / 1e9,
                                     "tile_GBps": float(k_by.sum() / (k_ms.sum() / 1e3) / 1e9) if len(k_ms) else None}
        if name == "c64":
            ca = Q.circuit_from(circ).finalize(dt)
            best = ca.autotune(s, reps=2)
            s.set_basis(0)
            ca.apply(s)
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(args.steps):
                s.set_basis(0)
                ca.apply(s)
            t1.record()
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / args.steps
            out["c64_autotuned"] = {"gates_per_s": G / (ms / 1e3), "ms": ms, "passes": ca.info()["passes"],
                                    "tile_bits": best["tile_bits"], "low_bits": best["low_bits"]}
        out[f"{name}_sum_z"] = Q.expectation(s, H)
        del s
        torch.cuda.empty_cache()
    line = {"metric": "random-circuit gates/s (28 qubits, 500 gates)", "value": out["c64_fused"]["gates_per_s"],
            "unit": "gates/s", "n_gpus": 1, "steps": args.steps, "higher_is_better": True, "dtype": "f32/f64",
            "data": "synthetic", "config": {"workload": f"{n}-qubit random circuit, {G} gates, seed 2"}, "detail": out}
    print(json.dumps(line), flush=True)


def gnn_flops(graphs, H=64, L=3, O=8):
    """Algorithmic FP32 flops of one forward and one backward launch over
    `graphs` (multiply-add = 2): neighbour means, the two H x d products per
    node and layer, readout and MLP; the backward recomputes the forward and
    adds the weight-gradient and input-gradient products."""
    fwd = bwd = 0.0
    for n, e in graphs:
        adj = 2 * len(e)
        f = n * H + 2 * H * H + 2 * O * H
        b = 2 * O * H + 4 * H * H
        d = 2
        for l in range(L):
            f += adj * d + 4 * n * H * d
            b += adj * d + 4 * n * H * d + (4 * n * H * H + adj * H if l > 0 else 0)
            d = H
        fwd += f
        bwd += f + b
    return fwd, bwd


def fp32_alu_peak_tflops(sm_mhz):
    """FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def run_gnn_workload(args):
    """Learned-initialiser network: 256 graphs of 26 nodes (half 3-regular, half
    Erdos-Renyi G(26, 0.3), seed 5), hidden 64, 3 layers, 8 outputs; one training
    step = forward + MSE + backward + Adam, all device kernels."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build, inputs as I
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    from paper_2406_17248_gb300.qaoa_init import Initialiser
    graphs = I.graph_set(256, 5, (26, 26))
    gb = Q.Graphs.from_graphs(graphs)
    init = Initialiser(p=4, seed=5)
    net = init.net
    y = torch.zeros(len(graphs), 8, dtype=torch.float32, device="cuda")
    t = torch.randn_like(y)
    dy = torch.zeros_like(y)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grad = torch.zeros(net.n_weights, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def step():
        net.train_step(gb, t, 1e-4, loss)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    reps = max(args.steps, 10) * 200
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    clocks = ClockSampler()
    clocks.start()
    ev[0].record(st)
    for _ in range(reps):
        net.forward(gb, y)
    ev[1].record(st)
    for _ in range(reps):
        net.backward(gb, dy, grad)
    ev[2].record(st)
    for _ in range(reps):
        step()
    ev[3].record(st)
    torch.cuda.synchronize()
    ck = clocks.stop()
    fwd_us = 1e3 * ev[0].elapsed_time(ev[1]) / reps
    bwd_us = 1e3 * ev[1].elapsed_time(ev[2]) / reps
    step_us = 1e3 * ev[2].elapsed_time(ev[3]) / reps
    f_fl, b_fl = gnn_flops(graphs)
    sm = ck.get("sm_max_mhz") or 2070
    peak = fp32_alu_peak_tflops(sm)
    dom = "backward" if bwd_us >= fwd_us else "forward"
    ach = (b_fl / (bwd_us * 1e-6) if dom == "backward" else f_fl / (fwd_us * 1e-6)) / 1e12
    # end to end through the public API: graphs and targets from the host, loss back
    tgt_h = torch.randn(len(graphs), 8, dtype=torch.float32).pin_memory()
    loss_h = torch.zeros(1, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    e2e_reps = 20
    for _ in range(e2e_reps):
        gbh = Q.Graphs.from_graphs(graphs)
        t.copy_(tgt_h, non_blocking=True)
        net.train_step(gbh, t, 1e-4, loss)
        loss_h.copy_(loss, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - h0) / e2e_reps
    no, ao, adj = I.pack_graphs(graphs)
    line = {"metric": "GNN initialiser training step (forward+MSE+backward+Adam, two launches), graphs/s",
            "value": len(graphs) / (step_us * 1e-6), "unit": "graphs/s", "n_gpus": 1, "steps": reps,
            "warmup": max(3, args.warmup), "ms_per_step": step_us / 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights, f32 arithmetic", "data": "synthetic",
            "config": {"workload": "256 graphs x 26 nodes (3-regular / G(26,0.3)), hidden 64, 3 layers, 8 outputs, "
                                   "seed 5", "l2": "inputs (1 MB) are L2-resident; latency-bound launches"},
            "forward_us": fwd_us, "backward_us": bwd_us, "step_us": step_us,
            "roofline": {"bound": "alu", "kernel": f"gnn_{dom}_kernel", "achieved": ach, "peak": peak,
                         "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                         "peak_note": f"FP32 FMA: 152 SMs x 128 lanes x 2 x {sm} MHz"},
            "e2e": {"value": len(graphs) / e2e_s, "unit": "graphs/s",
                    "h2d_bytes_per_step": int(4 * (no.size + ao.size + adj.size) + tgt_h.numel() * 4),
                    "d2h_bytes_per_step": 4},
            "gpu_launches": reps * (1 + 2 + 2), "clocks": ck}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = gnn_cpu_baseline(graphs, net)
    print(json.dumps(line), flush=True)


def gnn_cpu_baseline(graphs, net):
    """The FP64 oracle's forward+backward on a bounded sample of the same graphs."""
    import numpy as np
    from oracle import gnn_oracle as G
    from paper_2406_17248_gb300 import inputs as I
    _, wb = net.get_weights()
    w = (wb.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    sample = graphs[:16]
    batch = I.pack_graphs(sample)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < 10.0:
        y = G.forward(w, *batch)
        _, dy = G.mse(y, np.zeros_like(y))
        G.backward(w, *batch, dy)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k * len(sample) / dt, "unit": "graphs/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} x {len(sample)} graphs of 26 nodes, forward + MSE + backward (no Adam)"}


def run_dense_workload(args):
    """Dense k-qubit blocks on 28 qubits complex64 (2 GiB): a seeded random
    unitary on spread targets, tensor cores (tcgen05) vs CUDA cores."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build, inputs as I
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    n = args.n if args.n != 30 else 28
    k = args.block_k
    targets = [0, 9, 17, 22, n - 1, 13][:k]
    rng = np.random.default_rng(k)
    U = np.linalg.qr(rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k)))[0]
    s = Q.State(n, Q.C64).set_plus()
    st = torch.cuda.current_stream()
    res = {}
    clocks = ClockSampler()
    for eng, name in ((2, "tensor"), (1, "cuda_core")):
        for _ in range(max(3, args.warmup)):
            Q.apply_matrix(s, targets, U, eng)
        torch.cuda.synchronize()
        if eng == 2:
            clocks.start()
        Q.trace_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            Q.apply_matrix(s, targets, U, eng)
        e1.record(st)
        torch.cuda.synchronize()
        Q.trace_enable(False)
        if eng == 2:
            ck = clocks.stop()
        k_ms, k_by, _ = Q.trace_read()
        res[name] = {"ms_per_block": e0.elapsed_time(e1) / args.steps, "kernel_ms": float(np.mean(k_ms)),
                     "kernel_GBps": float(np.mean(k_by) / (np.mean(k_ms) / 1e3) / 1e9)}
    peak, peak_kind = measured_peak_hbm()
    tc = res["tensor"]
    tflops = 3 * 8 * (1 << k) * (1 << n) / (tc["kernel_ms"] / 1e3) / 1e12
    # end to end: the state from pinned host memory, the block, the state back
    h = torch.empty(1 << n, dtype=torch.complex64).pin_memory()
    h.copy_(s.amplitudes, non_blocking=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        s.amplitudes.copy_(h, non_blocking=True)
        Q.apply_matrix(s, targets, U, 2)
        h.copy_(s.amplitudes, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / 2
    line = {"metric": f"dense {k}-qubit block applications/s, {n} qubits complex64 (tcgen05 tensor cores)",
            "value": 1e3 / tc["ms_per_block"], "unit": "blocks/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": tc["ms_per_block"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (tf32 head/tail split)", "data": "synthetic",
            "config": {"workload": f"{n}-qubit complex64 state, seeded random {k}-qubit unitary on qubits {targets}",
                       "l2": "state 2 GiB > L2, no flush needed"},
            "roofline": {"bound": "hbm", "kernel": "dense_ws_kernel<5>" if k == 5 else f"dense_tc_kernel<{k}>", "achieved": tc["kernel_GBps"], "peak": peak,
                         "unit": "GB/s", "frac": tc["kernel_GBps"] / peak, "traffic": None,
                         "peak_kind": f"{peak_kind} hbm_gbs", "tensor_tflops": tflops},
            "cuda_core": res["cuda_core"], "tensor": tc,
            "e2e": {"value": 1.0 / e2e_s, "unit": "blocks/s", "h2d_bytes_per_step": 8 << n,
                    "d2h_bytes_per_step": 8 << n},
            "gpu_launches": 2 * args.steps, "clocks": ck}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = dense_cpu_baseline(k, U, targets, n)
    print(json.dumps(line), flush=True)


def dense_cpu_baseline(k, U, targets, n, n_small=20):
    """The oracle's block applier on a 20-qubit state, scaled by 2^(20 - n)."""
    import numpy as np
    from oracle import qsim_oracle as O
    from paper_2406_17248_gb300 import inputs as I
    psi = I.random_state(n_small, 1)
    tg = [t % n_small for t in targets]
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < 10.0:
        psi = O.apply_gate(psi, n_small, U, tg)
        reps += 1
    dt = time.perf_counter() - t0
    return {"value": reps / dt * 2.0 ** (n_small - n), "unit": "blocks/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} applications at {n_small} qubits (complex128 numpy), scaled by 2^({n_small}-{n})"}


def run_hea_workload(args):
    """12-qubit HEA, 4 layers (RY, RZ per qubit, open CNOT ladder), 96 parameters
    U[-pi, pi] seed 1, H = sum Z_i Z_{i+1} + 0.5 sum X_i, complex128 from |0>:
    energy + 96 gradients per evaluation.  Single: one parameter vector through
    the fused tile engine; many: 1024 parameter vectors (seeds 1..1024) in one
    batched launch (each instance's psi and lam in one CTA's shared memory)."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build, inputs as I
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    n, layers = (args.n if args.n != 30 else 12), 4
    circ = I.hea_circuit(n, layers)
    ham = I.chain_zz_x(n, 0.5)
    params = I.uniform_params(circ.n_params, 1)
    c = Q.circuit_from(circ).finalize(Q.C128)
    h = Q.Hamiltonian(ham)
    psi, lam = Q.State(n, Q.C128), Q.State(n, Q.C128)
    for _ in range(max(3, args.warmup)):
        psi.set_basis(0)
        Q.expectation_with_grad(psi, lam, c, h, params)
    torch.cuda.synchronize()
    reps = max(args.steps, 10) * 10
    t0 = time.perf_counter()
    for _ in range(reps):
        psi.set_basis(0)
        E, G = Q.expectation_with_grad(psi, lam, c, h, params)
    torch.cuda.synchronize()
    single = reps / (time.perf_counter() - t0)
    n_inst = 1024
    inst = [I.Instance(circ, ham, I.uniform_params(circ.n_params, s)) for s in range(1, n_inst + 1)]
    b = Q.Batch(inst, Q.C128)
    pd = torch.tensor(np.concatenate([it.params for it in inst]), dtype=torch.float64, device="cuda")
    ed = torch.empty(n_inst, dtype=torch.float64, device="cuda")
    gd = torch.empty_like(pd)
    for _ in range(max(3, args.warmup)):
        b.expectation_with_grad_device(pd, ed, gd)
    clocks = ClockSampler()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        b.expectation_with_grad_device(pd, ed, gd)
    ev1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    many = n_inst / (ms / 1e3)
    line = {"metric": "12q HEA c128 adjoint energy+grad evals/s (one vector; 1024 vectors batched)",
            "value": many, "unit": "evals/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "12-qubit HEA, 4 layers, 96 params U[-pi,pi] (seed 1; batch seeds 1..1024), "
                                   "H = sum ZZ + 0.5 sum X, complex128", "l2": "64 KiB states: shared-memory bound"},
            "single_vector": {"value": single, "unit": "evals/s", "engine": "fused tile passes, one call per eval"},
            "batched": {"value": many, "unit": "evals/s", "instances": n_inst},
            "energy_single": E, "gpu_launches": args.steps, "clocks": ck}
    if not args.no_cpu_baseline:
        from oracle import qsim_oracle as O
        E0, G0 = O.adjoint_gradient(circ, ham, params, O.zero_state(n))
        line["error_vs_oracle"] = {"energy": abs(E - E0), "grad_max": float(np.max(np.abs(G - G0)))}
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 10.0:
            O.adjoint_gradient(circ, ham, params, O.zero_state(n))
            k += 1
        line["cpu_baseline"] = {"value": k / (time.perf_counter() - t0), "unit": "evals/s", "cores": 1,
                                "kind": "oracle", "sample": f"{k} oracle adjoint evaluations of the same instance"}
    print(json.dumps(line), flush=True)


def run_dm_workload(args):
    """Noisy 14-qubit HEA (4 layers) as a density matrix (a 28-qubit complex64
    vector, 2 GiB): depolarizing p = 0.01 on every qubit after every layer, then
    tr(rho H) with H = sum ZZ + 0.5 sum X.  A step = one noisy evolution from
    |0><0| plus the expectation."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build, inputs as I
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    n, layers = 14, 4
    circ = I.hea_circuit(n, layers)
    params = I.uniform_params(circ.n_params, 1)
    layer_end = [i for i, g in enumerate(circ.gates) if g.kind == "X" and g.targets == (n - 1,)]
    ch = {i: [("depolarizing", (0.01,), q) for q in range(n)] for i in layer_end}
    c = Q.dm_circuit_from(circ, ch).finalize(Q.C64)
    H = Q.Hamiltonian(I.chain_zz_x(n, 0.5))
    s = Q.State(2 * n, Q.C64)
    st = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        s.set_basis(0)
        c.apply(s, params)
        E = Q.dm_expectation(s, H)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    Q.trace_enable(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_basis(0)
        c.apply(s, params)
        E = Q.dm_expectation(s, H)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / args.steps
    Q.trace_enable(False)
    ck = clocks.stop()
    k_ms, k_by, k_kind = Q.trace_read()
    peak, peak_kind = measured_peak_hbm()
    ach = float(k_by.sum() / (k_ms.sum() / 1e3) / 1e9)
    # the passes' kernels by traced time (compiled per circuit, library micro-op, interpreter)
    kinds = {int(k): float(k_ms[k_kind == k].sum()) for k in np.unique(k_kind)} if len(k_ms) else {}
    top = Q.TRACE_KINDS.get(max(kinds, key=kinds.get), "?") if kinds else None
    line = {"metric": "noisy density-matrix evolutions + tr(rho H)/s, 14 qubits (28-qubit vector) complex64",
            "value": 1.0 / wall, "unit": "evals/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "14-qubit HEA, 4 layers, params U[-pi,pi] seed 1, depolarizing 0.01 on every "
                                   "qubit after every layer; H = sum ZZ + 0.5 sum X", "l2": "2 GiB state > L2"},
            "energy": E, "passes": c.info()["passes"],
            "roofline": {"bound": "hbm", "kernel": top, "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": None, "peak_kind": f"{peak_kind} hbm_gbs"},
            "pass_kernels_ms": {Q.TRACE_KINDS.get(k, str(k)): v / max(args.steps, 1) for k, v in kinds.items()},
            "gpu_launches": int(len(k_ms) / max(args.steps, 1)) + 3, "clocks": ck}
    if not args.no_cpu_baseline:
        from oracle import dm_oracle as D
        n_s = 6
        cs = I.hea_circuit(n_s, layers)
        ps = I.uniform_params(cs.n_params, 1)
        le = [i for i, g in enumerate(cs.gates) if g.kind == "X" and g.targets == (n_s - 1,)]
        chs = {i: [("depolarizing", (0.01,), q) for q in range(n_s)] for i in le}
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 10.0:
            D.expectation(D.run(cs, ps, chs, n_s), I.chain_zz_x(n_s, 0.5))
            k += 1
        line["cpu_baseline"] = {"value": k / (time.perf_counter() - t0), "unit": "evals/s", "cores": 1,
                                "kind": "oracle", "sample": f"{k} dense-matrix oracle evaluations at 6 qubits "
                                                            "(not scaled: the dense oracle grows as 8^n)"}
    print(json.dumps(line), flush=True)


def run_dcqaoa_workload(args):
    """DC-QAOA on the 12-qubit longitudinal-field Ising chain (J = h = 1, k = 0),
    one layer (gamma, beta, alpha), CD term sum Y: ``--instances`` random starts
    U[0, 0.1) (seeds 1, 2, ...) trained together with Adam (lr 0.05).  A step =
    one batched energy + adjoint gradient of every start (complex128, each
    start's psi and lam in one CTA's shared memory) and one Adam kernel over all
    parameters.  value = start-steps/s."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build, inputs as I
    build.build()
    from paper_2406_17248_gb300 import qsim as Q, vqa
    n, p = 12, 1
    starts = args.instances
    inst = vqa.dcqaoa_multistart(n, p, starts, seed=1)
    res = {}
    for dt, name in ((Q.C64, "c64"), (Q.C128, "c128")):
        opt = vqa.BatchAdam(inst, dt, lr=0.05)
        for _ in range(max(3, args.warmup)):
            opt.step()
        torch.cuda.synchronize()
        clocks = ClockSampler()
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            opt.step()
        ev1.record()
        torch.cuda.synchronize()
        ck = clocks.stop()
        ms = ev0.elapsed_time(ev1) / args.steps
        res[name] = {"ms": ms, "value": starts / (ms / 1e3), "clocks": ck}
    # the optimisation itself (untimed): 100 more steps of the complex128 run
    opt.run(max(1, 100 - opt.t))
    e_final = opt.energies.cpu().numpy()
    # end to end through the public call with host buffers: params H2D, energies
    # and gradients D2H every step, Adam on the host
    b = opt.batch
    x = np.concatenate([it.params for it in inst])
    m, v = np.zeros_like(x), np.zeros_like(x)
    b.expectation_with_grad(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in range(1, args.steps + 1):
        e, g = b.expectation_with_grad(x)
        gc = np.concatenate(g)
        m = 0.9 * m + 0.1 * gc
        v = 0.999 * v + 0.001 * gc * gc
        x = x - 0.05 * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
    e2e_s = (time.perf_counter() - t0) / args.steps
    line = {"metric": "DC-QAOA multistart Adam start-steps/s (12-qubit LFIM, p = 1, energy + 3 gradients + update)",
            "value": res["c128"]["value"], "unit": "start-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": res["c128"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"DC-QAOA, 12-qubit Ising chain J = h = 1, k = 0, p = 1, CD term sum Y, "
                                   f"{starts} starts U[0, 0.1) seeds 1..{starts}, Adam lr 0.05, complex128",
                       "starts": starts, "l2": "states in shared memory; L2 not involved"},
            "c64": {"value": res["c64"]["value"], "unit": "start-steps/s", "ms_per_step": res["c64"]["ms"]},
            "after_training": {"adam_steps": opt.t, "min_energy": float(e_final.min()), "ground_energy": -23.0,
                                "starts_within_1e-3": int((e_final < -23.0 + 1e-3).sum())},
            "e2e": {"value": starts / e2e_s, "unit": "start-steps/s", "h2d_bytes_per_step": int(x.nbytes),
                    "d2h_bytes_per_step": int(x.nbytes + 8 * starts)},
            "gpu_launches": 2 * args.steps, "clocks": res["c128"]["clocks"]}
    if not args.no_cpu_baseline:
        from oracle import gnn_oracle as G
        from oracle import qsim_oracle as O
        it = inst[0]
        xs = np.array(it.params)
        ms_, vs_ = np.zeros_like(xs), np.zeros_like(xs)
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 10.0:
            k += 1
            e, g = O.adjoint_gradient(it.circuit, it.ham, xs, O.zero_state(n))
            xs, ms_, vs_ = G.adam(xs, ms_, vs_, g, k, 0.05)
        line["cpu_baseline"] = {"value": k / (time.perf_counter() - t0), "unit": "start-steps/s", "cores": 1,
                                "kind": "oracle", "sample": f"{k} oracle Adam steps of start 1"}
    print(json.dumps(line), flush=True)


def run_traj_workload(args):
    """Noisy n-qubit HEA (``--n``, default 12; 4 layers, 8n parameters U[-pi, pi]
    seed 1) with a depolarizing channel p = 0.01 on every qubit after every layer
    (4n sites), H = sum ZZ + 0.5 sum X, complex64, by Monte-Carlo trajectories:
    a step = ``--instances`` trajectories, each with its energy and adjoint
    gradient, and the mean gradient.  value = trajectories/s.  Up to 13 qubits
    each trajectory runs in one CTA's shared memory; beyond, one trajectory at a
    time on the fused tile passes.  Up to 13 qubits the exact tr(rho H) of the
    same noisy circuit through the density-matrix engine is timed beside it."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import build, inputs as I
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    n, layers = (args.n if args.n != 30 else 12), 4
    circ = I.hea_circuit(n, layers)
    params = I.uniform_params(circ.n_params, 1)
    ham = I.chain_zz_x(n, 0.5)
    layer_end = [i for i, g in enumerate(circ.gates) if g.kind == "X" and g.targets == (n - 1,)]
    ch = {i: [("depolarizing", (0.01,), q) for q in range(n)] for i in layer_end}
    n_t = args.instances
    eng = Q.trajectories_from(circ, ch, Q.C64)
    H = Q.Hamiltonian(ham)
    pd = torch.tensor(params, dtype=torch.float64, device="cuda")
    ed = torch.empty(n_t, dtype=torch.float64, device="cuda")
    gd = torch.empty(circ.n_params, dtype=torch.float64, device="cuda")
    for w in range(max(3, args.warmup)):
        eng.run_device(H, pd, n_t, seed=7, energies=ed, grad_mean=gd, first=w * n_t)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for s in range(args.steps):
        eng.run_device(H, pd, n_t, seed=7, energies=ed, grad_mean=gd, first=(s + 8) * n_t)
    ev1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    e = ed.cpu().numpy()
    launches = 2 * args.steps  # shared-memory engine: the trajectory kernel and the row mean
    if eng.info()["grid_grad"] == 0:
        # one trajectory at a time: count the traced fused-pass launches of one
        # more (untimed) step; their set-up, Hamiltonian and reduction kernels
        # come on top
        Q.trace_enable(True)
        eng.run_device(H, pd, n_t, seed=7, energies=ed, grad_mean=gd, first=99 * n_t)
        torch.cuda.synchronize()
        Q.trace_enable(False)
        launches = len(Q.trace_read()[0]) * args.steps
    # end to end through the host-buffer call (params H2D, energies + gradient D2H)
    eng.run(H, params, n_t, seed=7, first=99 * n_t, grad=True)
    t0 = time.perf_counter()
    for s in range(args.steps):
        eh, gh = eng.run(H, params, n_t, seed=7, first=(s + 100) * n_t, grad=True)
    e2e_s = (time.perf_counter() - t0) / args.steps
    # exact noisy energy through the density-matrix engine (a 2n-qubit vector)
    dm = None
    if n <= 13:
        dmc = Q.dm_circuit_from(circ, ch).finalize(Q.C64)
        rho = Q.State(2 * n, Q.C64)
        rho.set_basis(0)
        dmc.apply(rho, params)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            rho.set_basis(0)
            dmc.apply(rho, params)
            exact = Q.dm_expectation(rho, H)
        dm = {"energy": exact, "seconds_per_eval": (time.perf_counter() - t0) / 5,
              "state": f"{2 * n}-qubit complex64 vector"}
    info = eng.info()
    line = {"metric": f"noisy VQE Monte-Carlo trajectories/s ({n}-qubit HEA, energy + {circ.n_params}-parameter "
                      "adjoint gradient each)",
            "value": n_t / (ms / 1e3), "unit": "trajectories/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n}-qubit HEA, 4 layers, params U[-pi,pi] seed 1, depolarizing 0.01 on every "
                                   f"qubit after every layer ({4 * n} sites), H = sum ZZ + 0.5 sum X, complex64, "
                                   f"{n_t} trajectories per step", "trajectories": n_t,
                       "engine": "shared memory, many trajectories per launch" if info["grid_grad"] > 0
                       else "fused tile passes, one trajectory at a time",
                       "l2": "states in shared memory; L2 not involved" if info["grid_grad"] > 0
                       else f"state 2^{n} x 8 B per trajectory"},
            "mean_energy": float(e.mean()), "std_error": float(e.std() / np.sqrt(e.size)),
            "density_matrix": dm,
            "e2e": {"value": n_t / e2e_s, "unit": "trajectories/s", "h2d_bytes_per_step": int(params.nbytes),
                    "d2h_bytes_per_step": int(8 * n_t + params.nbytes)},
            "grid": info["grid_grad"], "gpu_launches": launches, "clocks": ck}
    if not args.no_cpu_baseline:
        from oracle import traj_oracle as T
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 10.0:
            T.trajectory_energy_and_grad(circ, ham, params, ch, 7, k)
            k += 1
        line["cpu_baseline"] = {"value": k / (time.perf_counter() - t0), "unit": "trajectories/s", "cores": 1,
                                "kind": "oracle", "sample": f"{k} oracle trajectories (energy + adjoint gradient)"}
    print(json.dumps(line), flush=True)


def measure_gate_sweep(Q, n, dt, reps):
    """Single-gate sweep on an n-qubit state from |+>^n: H, RZ(0.3), CNOT (control
    q + 1) and CZ (control q + 1) on every target q, each gate one launch of the
    per-gate kernels (`fuse = -1`), CUDA events on the launching stream.
    Algorithmic bytes count the amplitudes a gate changes, read and written: H and
    RZ 2 S, CNOT S, CZ S / 2 (S = the state's bytes)."""
    import numpy as np
    import torch
    from paper_2406_17248_gb300 import inputs as I
    S = (8 if dt == Q.C64 else 16) * float(1 << n)
    s = Q.State(n, dt)
    s.set_plus()
    kinds = {"H": (lambda q: I.Gate("H", (q,)), 2 * S), "RZ": (lambda q: I.Gate("RZ", (q,), const=0.3), 2 * S),
             "CNOT": (lambda q: I.Gate("X", (q,), ((q + 1) % n,)), S),
             "CZ": (lambda q: I.Gate("Z", (q,), ((q + 1) % n,)), S / 2)}
    circs = {k: [Q.circuit_from(I.Circuit(n, [mk(q)])).finalize(dt, fuse=-1) for q in range(n)]
             for k, (mk, _) in kinds.items()}
    st = torch.cuda.current_stream()
    for k in kinds:
        for q in range(n):
            circs[k][q].apply(s, [])
    torch.cuda.synchronize()
    peak, peak_kind = measured_peak_hbm()
    per = {}
    tot_bytes = tot_ms = 0.0
    for k, (_, by) in kinds.items():
        ms_q = []
        for q in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                circs[k][q].apply(s, [])
            e1.record(st)
            e1.synchronize()
            ms_q.append(e0.elapsed_time(e1) / reps)
        gbs = [by / (m / 1e3) / 1e9 for m in ms_q]
        per[k] = {"GBps_median": float(np.median(gbs)), "GBps_min": float(np.min(gbs)),
                  "frac_median": float(np.median(gbs)) / peak, "frac_min": float(np.min(gbs)) / peak,
                  "ms_median": float(np.median(ms_q)), "GBps_by_target": [round(g, 1) for g in gbs]}
        tot_bytes += by * n
        tot_ms += sum(ms_q)
    del s
    torch.cuda.empty_cache()
    ach = tot_bytes / (tot_ms / 1e3) / 1e9
    return {"n_qubits": n, "dtype": "complex64" if dt == Q.C64 else "complex128", "GBps": ach, "peak": peak,
            "frac": ach / peak, "peak_kind": f"{peak_kind} hbm_gbs", "ms": tot_ms, "gates_per_s": 4 * n / (tot_ms / 1e3),
            "launches": 4 * n * reps, "per_kind": per}


def run_gates_workload(args):
    """`measure_gate_sweep` at --n qubits (default 30), complex64 or complex128."""
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim as Q
    dt = Q.C128 if args.gate_dtype == "c128" else Q.C64
    reps = max(1, args.steps)
    clocks = ClockSampler()
    clocks.start()
    r = measure_gate_sweep(Q, args.n, dt, reps)
    ck = clocks.stop()
    line = {"metric": f"{args.n}-qubit {r['dtype']} single-gate sweep (H, RZ, CNOT, CZ on every qubit), HBM GB/s",
            "value": r["GBps"], "unit": "GB/s", "n_gpus": 1, "steps": reps, "warmup": 1,
            "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if dt == Q.C64 else "f64", "data": "synthetic",
            "config": {"workload": f"{args.n} qubits from |+>^n, 4 x {args.n} single-gate launches", "l2": "state > L2"},
            "gates_per_s": r["gates_per_s"],
            "roofline": {"bound": "hbm", "achieved": r["GBps"], "peak": r["peak"], "unit": "GB/s", "frac": r["frac"],
                         "traffic": None, "peak_kind": r["peak_kind"]},
            "per_kind": r["per_kind"], "gpu_launches": r["launches"], "clocks": ck}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="qaoa30", choices=["qaoa30", "batch", "random28", "gnn", "dense28", "hea12", "dm14", "dcqaoa12", "traj12", "gates"])
    ap.add_argument("--instances", type=int, default=2048)
    ap.add_argument("--plain-instances", type=int, default=2048)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--low-bits", type=int, default=0)
    ap.add_argument("--cpu-qubits", type=int, default=24)
    ap.add_argument("--ref-qubits", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="default workload: skip the gate sweep and batch lines")
    ap.add_argument("--block-k", type=int, default=5)
    ap.add_argument("--gate-dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--checkpoint", type=int, default=0, help="QAOA: adjoint state checkpoints every K layers")
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch_workload(args)
    if args.workload == "dm14":
        return run_dm_workload(args)
    if args.workload == "dcqaoa12":
        return run_dcqaoa_workload(args)
    if args.workload == "traj12":
        return run_traj_workload(args)
    if args.workload == "gates":
        return run_gates_workload(args)
    if args.workload == "hea12":
        return run_hea_workload(args)
    if args.workload == "dense28":
        return run_dense_workload(args)
    if args.workload == "gnn":
        return run_gnn_workload(args)
    if args.workload == "random28":
        if args.n == 30:
            args.n = 28
        return run_random_workload(args)
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
