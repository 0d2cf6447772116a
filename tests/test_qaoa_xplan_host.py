"""Host-side check of the complex64 two-shape QAOA plan (no GPU): the passes,
phases, coefficient offsets and output slots that qs_qaoa_xplan reports are
replayed in FP64 on a numpy state, one operation per phase step exactly as the
kernels define them, and the resulting energy and gradients are compared with
the oracle's adjoint evaluation (§5.2 ansatz, §6.2 QuPack interface).  A
planner mistake (a mixer qubit skipped or applied twice, a cost layer out of
order, a wrong coefficient offset or slot) changes the result."""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2406_17248_gb300 import inputs as I


@pytest.fixture(scope="module")
def Q():
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def _coef_table(n_edges, gamma, beta, gs):
    """Per layer: lut[k] = exp(-i gs gamma C), C = |E| - 2k, its conjugate, and
    the RX coefficients (cos b/2, sin b/2) and (cos b/2, -sin b/2)."""
    tab = []
    for g, b in zip(gamma, beta):
        C = n_edges - 2.0 * np.arange(n_edges + 1)
        lut = np.exp(-1j * gs * g * C)
        tab += list(lut) + list(np.conj(lut))
        c, s = np.cos(0.5 * b), np.sin(0.5 * b)
        tab += [complex(c, s), complex(c, -s)]
    return np.array(tab)


def _rx(psi, n, q, c, s):
    """[[c, -is], [-is, c]] on qubit q."""
    v = psi.reshape(-1, 2, 1 << q)
    a0, a1 = v[:, 0, :].copy(), v[:, 1, :].copy()
    v[:, 0, :] = c * a0 - 1j * s * a1
    v[:, 1, :] = c * a1 - 1j * s * a0
    return v.reshape(-1)


def _gx(lam, psi, n, q):
    """Im <lam|X_q|psi>."""
    idx = np.arange(1 << n) ^ (1 << q)
    return float(np.imag(np.vdot(lam, psi[idx])))


def replay(plan, slots, n, edges, gamma, beta, gs, p):
    """Run the plan's steps on FP64 states and gather the outputs by slot."""
    tab = _coef_table(len(edges), gamma, beta, gs)
    C = O.cut_values(n, edges).astype(np.int64)  # C(x) = sum over edges of z_a z_b
    cut = (len(edges) - C) // 2  # edges cut by x: the LUT index
    psi = np.zeros(1 << n, complex)
    lam = np.zeros(1 << n, complex)
    vals = np.zeros(len(slots))
    for P in plan:
        acc = [0.0, 0.0, 0.0]
        two = P["two"]
        if P["flags"] & 1:
            psi = O.plus_state(n).astype(complex)
        if two and P["flags"] & 2:
            lam = np.zeros(1 << n, complex)
        c1 = tab[P["c1"]] if P["c1"] >= 0 else 1.0
        c3 = tab[P["c3"]] if P["c3"] >= 0 else 1.0
        seen1, seen3 = set(), set()
        R = 3 if two else 4  # register bits per phase (psi/lam kernel: 3)
        for ph in P["phases"]:
            reg = ph["reg"][:R]
            assert len(set(reg)) == R and all(q >= 0 for q in reg) and all(q == -1 for q in ph["reg"][R:])
            assert all((P["S"] >> q) & 1 for q in reg)
            for step, mask, cf, grad_flag, seen in ((0, ph["m1"], c1, 8, seen1), (2, ph["m3"], c3, 16, seen3)):
                if step == 2:  # the diagonal step sits between the two mixer steps
                    d = ph["diag"]
                    if d == 1:
                        psi = psi * tab[P["cd"] + cut]
                    elif d == 2:
                        acc[1] += float(np.sum(C * np.imag(np.conj(lam) * psi)))
                        lut = tab[P["cd"] + cut]
                        psi, lam = psi * lut, lam * lut
                    elif d == 3:
                        acc[1] += float(np.sum(C * np.abs(psi) ** 2))
                        if two:
                            lam = C * psi
                for r in range(R):
                    if not (mask >> r) & 1:
                        continue
                    q = ph["reg"][r]
                    assert q not in seen, "a mixer qubit taken twice in one pass step"
                    seen.add(q)
                    if two and P["flags"] & grad_flag:
                        acc[step] += _gx(lam, psi, n, q)
                    psi = _rx(psi, n, q, cf.real, cf.imag)
                    if two:
                        lam = _rx(lam, n, q, cf.real, cf.imag)
        for k in range(3):
            if P["slot"][k] >= 0:
                vals[P["slot"][k]] += acc[k]
    out = np.zeros(1 + 2 * p)
    for s, (o, w) in enumerate(slots):
        out[o] += w * vals[s]
    return out, psi


CASES = [(12, 1, 9, 2, 0.5), (13, 3, 9, 2, 1.0), (14, 2, 9, 3, 0.5), (16, 4, 10, 3, 0.5), (17, 2, 11, 3, 1.0)]


@pytest.mark.parametrize("n,p,tb,lb,gs", CASES)
def test_gradient_plan_replays_to_the_oracle(Q, n, p, tb, lb, gs):
    edges = I.random_regular_graph(n, 3 if n % 2 == 0 else 4, seed=n + 100 * p)
    ang = I.uniform_params(2 * p, n + p, 0.0, np.pi)
    gamma, beta = ang[:p], ang[p:]
    plan, slots = Q.qaoa_xplan(n, edges, p, gs, tb, lb, which=0)
    out, _ = replay(plan, slots, n, edges, gamma, beta, gs, p)
    E0, dg0, db0 = O.qaoa_expectation_with_grad(n, edges, gamma, beta, gs)
    assert abs(out[0] - E0) < 1e-10
    assert np.abs(out[1:1 + p] - dg0).max() < 1e-10
    assert np.abs(out[1 + p:] - db0).max() < 1e-10


@pytest.mark.parametrize("n,p,tb,lb,gs", CASES[:3])
def test_energy_plan_replays_to_the_oracle(Q, n, p, tb, lb, gs):
    edges = I.random_regular_graph(n, 3 if n % 2 == 0 else 4, seed=n)
    ang = I.uniform_params(2 * p, 7, 0.0, np.pi)
    plan, slots = Q.qaoa_xplan(n, edges, p, gs, tb, lb, which=1)
    out, psi = replay(plan, slots, n, edges, ang[:p], ang[p:], gs, p)
    E0, _, _ = O.qaoa_expectation_with_grad(n, edges, ang[:p], ang[p:], gs)
    assert abs(out[0] - E0) < 1e-10
    want = O.qaoa_layers_state(n, edges, ang[:p], ang[p:], gs)
    assert np.abs(psi - want).max() < 1e-12


def test_benchmark_plan_shape(Q):
    """30 qubits, p = 8: two passes per layer in both sweeps, every tile holds
    a qubit of small address stride (128-byte runs stream at full rate only
    then), at most six phases per pass."""
    n, p = 30, 8
    edges = I.random_regular_graph(n, 3, 3)
    plan, _ = Q.qaoa_xplan(n, edges, p, 0.5)
    fwd = [P for P in plan if P["two"] == 0]
    two = [P for P in plan if P["two"] == 1]
    assert len(fwd) == 2 * p and len(two) == 2 * p + 1
    for P in plan:
        assert P["n_phases"] <= 6
        elem = 16 if P["two"] else 8
        hi = [q for q in range(P["c"], n) if (P["S"] >> q) & 1]
        assert any((1 << q) * elem <= 16384 for q in hi), (P["S"], P["two"])


def _box_words(mp, n, S, toff):
    """Word indices that the tile's boxes deliver, in shared-memory order: a
    tiled tensor copy walks its box with dimension 0 fastest, box j of a tile
    starts at the word index of local offset j 2^lb (local bits ascend with the
    global ones)."""
    e, lb = mp["e"], mp["lb"]
    glob = [q for q in range(n) if (S >> q) & 1]
    m = len(glob)

    def l2g(l):
        return sum(1 << glob[i] for i in range(m) if (l >> i) & 1)

    out = []
    for j in range(1 << (m - lb)):
        wi = (toff + l2g(j << lb)) << e
        x = [(wi >> mp["a"][d]) & ((1 << mp["w"][d]) - 1) for d in range(5)]
        boxes = [1 << b for b in mp["box"]]
        idx = np.indices(boxes[::-1]).reshape(5, -1)[::-1]  # dimension 0 fastest
        addr = np.zeros(idx.shape[1], dtype=np.int64)
        for d in range(5):
            assert x[d] + boxes[d] <= (1 << mp["w"][d]), "box leaves its dimension"
            addr += (x[d] + idx[d]) << mp["a"][d]
        out.append(addr)
    return np.concatenate(out), e


@pytest.mark.parametrize("n,p,tb,lb", [(30, 8, 0, 0), (21, 3, 12, 3), (16, 2, 10, 3), (14, 2, 9, 2)])
def test_tile_tensor_maps_land_the_tile_in_local_order(Q, n, p, tb, lb):
    """Every pass's load and store maps move exactly the tile's words, each to
    the shared position of its local index, for the zero tile offset and for a
    random one (the complement bits set at random)."""
    edges = I.random_regular_graph(n, 3 if n % 2 == 0 else 4, seed=5)
    plan, _ = Q.qaoa_xplan(n, edges, p, 0.5, tb, lb)
    rng = np.random.default_rng(n)
    for P in plan:
        S = P["S"]
        glob = [q for q in range(n) if (S >> q) & 1]
        comp = [q for q in range(n) if not (S >> q) & 1]
        offs = [0, sum(1 << q for q in comp if rng.random() < 0.5)]
        for k, mp in enumerate(P["maps"]):
            assert mp["e"] == (1 if P["two"] and (k == 1 or not P["flags"] & 2) else 0)
            for toff in offs:
                got, e = _box_words(mp, n, S, toff)
                loc = np.arange(len(got)) >> e
                sub = np.arange(len(got)) & ((1 << e) - 1)
                want = np.zeros(len(got), dtype=np.int64)
                for i, q in enumerate(glob):
                    want += ((loc >> i) & 1) << q
                want = ((want + toff) << e) | sub
                assert len(got) == (1 << len(glob)) << e
                assert np.array_equal(got, want)


def _mix(v, n, q, t):
    """[[1, -it], [-it, 1]] on qubit q (the scaled mixer the kernels apply)."""
    w = v.reshape(-1, 2, 1 << q)
    a0, a1 = w[:, 0, :].copy(), w[:, 1, :].copy()
    w[:, 0, :] = a0 - 1j * t * a1
    w[:, 1, :] = a1 - 1j * t * a0
    return w.reshape(-1)


def replay_scaled(plan, slots, n, edges, tab, p):
    """The plan's steps in FP64 with the call's coefficient table exactly as the
    kernels use it: scaled mixers, renormalised LUTs, each mixer gradient term
    taken before its rotation and weighted by the phase weight times
    (1 + t^2)^-r after r rotations of its step."""
    C = O.cut_values(n, edges).astype(np.int64)
    cut = (len(edges) - C) // 2
    psi = np.zeros(1 << n, complex)
    lam = np.zeros(1 << n, complex)
    vals = np.zeros(len(slots))
    for P in plan:
        acc = [0.0, 0.0, 0.0]
        two = P["two"]
        if P["flags"] & 1:
            psi = O.plus_state(n).astype(complex)
        if two and P["flags"] & 2:
            lam = np.zeros(1 << n, complex)
        for k, ph in enumerate(P["phases"]):
            w1, w3 = tab[P["cw"] + 2 * k].real, tab[P["cw"] + 2 * k].imag
            wd = tab[P["cw"] + 2 * k + 1].real
            for step, mask, off, wgt in ((0, ph["m1"], P["c1"], w1), (2, ph["m3"], P["c3"], w3)):
                if step == 2:
                    d = ph["diag"]
                    if d == 1:
                        psi = psi * tab[P["cd"] + cut]
                    elif d == 2:
                        acc[1] += wd * float(np.sum(C * np.imag(np.conj(lam) * psi)))
                        lut = tab[P["cd"] + cut]
                        psi, lam = psi * lut, lam * lut
                    elif d == 3:
                        acc[1] += wd * float(np.sum(C * np.abs(psi) ** 2))
                        if two:
                            lam = C * psi
                qs = [ph["reg"][r] for r in range(4) if (mask >> r) & 1]
                if not qs:
                    continue
                t = tab[off].real
                kap = 1.0 / (1.0 + t * t)  # each scaled rotation multiplies |scale|^2 by 1 + t^2
                for r, q in enumerate(qs):
                    if two:
                        acc[step] += wgt * kap ** r * _gx(lam, psi, n, q)
                    psi = _mix(psi, n, q, t)
                    if two:
                        lam = _mix(lam, n, q, t)
        for k in range(3):
            if P["slot"][k] >= 0:
                vals[P["slot"][k]] += acc[k]
    out = np.zeros(1 + 2 * p)
    for s, (o, w) in enumerate(slots):
        out[o] += w * vals[s]
    return out, psi


# angles that put some layers in each mixer form (|cos b/2| >= |sin b/2| and <)
SCALED = [(12, 2, 9, 2, 0.5, (0.3, 2.9)), (13, 3, 9, 2, 1.0, (2.5, 0.4, 3.0)),
          (14, 2, 9, 3, 0.5, (2.2, 2.8)), (16, 4, 10, 3, 0.5, (0.2, 1.8, 2.7, -2.9))]


@pytest.mark.parametrize("n,p,tb,lb,gs,beta", SCALED)
def test_scaled_mixer_table_replays_to_the_oracle(Q, n, p, tb, lb, gs, beta):
    edges = I.random_regular_graph(n, 3 if n % 2 == 0 else 4, seed=n + 7)
    gamma = I.uniform_params(p, n, 0.0, np.pi)
    beta = np.array(beta)
    tab, _ = Q.qaoa_xcoef(n, edges, p, gamma, beta, gs, tb, lb)
    plan, slots = Q.qaoa_xplan(n, edges, p, gs, tb, lb, which=0)
    out, _ = replay_scaled(plan, slots, n, edges, tab, p)
    E0, dg0, db0 = O.qaoa_expectation_with_grad(n, edges, gamma, beta, gs)
    assert abs(out[0] - E0) < 1e-10
    assert np.abs(out[1:1 + p] - dg0).max() < 1e-9
    assert np.abs(out[1 + p:] - db0).max() < 1e-9


@pytest.mark.parametrize("n,p,tb,lb,gs,beta", SCALED)
def test_scaled_energy_plan_gives_the_state_up_to_the_reported_flip(Q, n, p, tb, lb, gs, beta):
    edges = I.random_regular_graph(n, 3 if n % 2 == 0 else 4, seed=n + 7)
    gamma = I.uniform_params(p, n + 1, 0.0, np.pi)
    beta = np.array(beta)
    tab, flip = Q.qaoa_xcoef(n, edges, p, gamma, beta, gs, tb, lb)
    assert flip == (int(np.sum(np.abs(np.sin(beta / 2)) > np.abs(np.cos(beta / 2)))) % 2 == 1)
    plan, slots = Q.qaoa_xplan(n, edges, p, gs, tb, lb, which=1)
    out, psi = replay_scaled(plan, slots, n, edges, tab, p)
    if flip:
        psi = psi[::-1]  # index NOT x = 2^n - 1 - x
    want = O.qaoa_layers_state(n, edges, gamma, beta, gs)
    assert np.abs(psi - want).max() < 1e-12
    E0, _, _ = O.qaoa_expectation_with_grad(n, edges, gamma, beta, gs)
    assert abs(out[0] - E0) < 1e-10
