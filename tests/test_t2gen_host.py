"""Host side of the per-circuit micro-op kernels (option fuse = 4): the
generator writes every phase of a plan as straight-line calls of the op bodies,
and the runtime compiler builds them for sm_103a, with no GPU needed
(qs_circuit_codegen).  Checks that the sources of the forward and adjoint plans
of mixed circuits (every op form, controls on register, tile and outside bits)
and of the random benchmark circuit compile, that each micro-op pass gets its
own kernel, and the argument checks."""
import re

import pytest

from paper_2406_17248_gb300 import inputs as I


@pytest.fixture(scope="module")
def Q():
    from paper_2406_17248_gb300 import build
    build.build()
    from paper_2406_17248_gb300 import qsim
    return qsim


def shared_param_circuit(n, seed):
    circ = I.random_mixed_circuit(n, 120, seed=seed, max_ctrls=2)
    gates = [I.Gate(g.kind, g.targets, g.ctrls, (g.param % 6) if g.param >= 0 else -1, g.coef, g.const, g.matrix)
             for g in circ.gates]
    return I.Circuit(n, gates, 6)


BODIES = ("t2_u1", "t2_r1", "t2_rx", "t2_x", "t2_z", "t2_neg_all", "t2_d1", "t2_d2", "t2_scale_all", "t2_u2",
          "t2_g1", "t2_g2", "t2_gd")


def test_mixed_circuits_generate_every_body_and_compile(Q):
    seen = set()
    for n, seed in ((14, 1), (17, 2)):
        circ = shared_param_circuit(n, seed)
        for which in (0, 1):
            r = Q.circuit_from(circ).codegen(which=which, compile=True)
            src = r["source"]
            assert r["passes"] >= 1 and r["cubin_bytes"] > 0
            # one kernel per micro-op pass, named by the pass index
            assert len(re.findall(r'extern "C" __global__', src)) == r["passes"]
            seen |= set(re.findall(r"(t2_[a-z0-9_]+)<", src))
            if which == 1:
                assert "c.grad(" in src  # adjoint passes accumulate 2 Re <lam|A|psi>
            else:
                assert "c.grad(" not in src
    assert set(BODIES) <= seen, set(BODIES) - seen


def test_random_benchmark_circuit_generates_every_pass(Q):
    circ = I.random_circuit(28, 500, seed=2)
    c = Q.circuit_from(circ)
    r = c.codegen(which=0, compile=True)
    assert r["passes"] == 11 and r["cubin_bytes"] > 0
    # CNOT controls outside the registers become predicated swaps
    assert "t2_x<1," in r["source"] and "if (((l0 &" in r["source"]


def test_codegen_argument_checks(Q):
    circ = shared_param_circuit(14, 3)
    c = Q.circuit_from(circ)
    with pytest.raises(Q.QSimError, match="INVALID_ARG"):
        c.codegen(which=2)
    with pytest.raises(Q.QSimError, match="INVALID_ARG"):
        c.codegen(fuse=-1)
    # the source alone, no compile: the same passes
    a = c.codegen(which=0, compile=False)
    b = c.codegen(which=0, compile=True)
    assert a["source"] == b["source"] and a["passes"] == b["passes"] and a["cubin_bytes"] == 0
    # a tile shape outside the micro-op form (complex64 needs >= 4 low bits): no kernels
    r = c.codegen(which=0, low_bits=2, tile_bits=10)
    assert r["passes"] == 0
