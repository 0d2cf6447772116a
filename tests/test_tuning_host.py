"""Autotuner cache bookkeeping on the host: keys depend on the gate structure,
the dtype, the qubit count and the GPU name but not on the angles; a hit skips
the tuner; entries survive a reload of the file."""
from paper_2406_17248_gb300 import inputs as I
from paper_2406_17248_gb300.tuning import TuneCache, structure_key


def test_structure_key():
    a = I.random_circuit(10, 50, 1)
    b = I.Circuit(10, [I.Gate(g.kind, g.targets, g.ctrls, g.param, g.coef, g.const + 0.5) for g in a.gates])
    assert structure_key(a, 0, "gpu") == structure_key(b, 0, "gpu")  # angles do not matter
    assert structure_key(a, 0, "gpu") != structure_key(a, 1, "gpu")
    assert structure_key(a, 0, "gpu") != structure_key(a, 0, "other")
    assert structure_key(a, 0, "gpu") != structure_key(I.random_circuit(10, 50, 2), 0, "gpu")


def test_cache_hits_skip_the_tuner(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def tune():
        calls.append(1)
        return {"tile_bits": 13, "low_bits": 2, "ms": 1.5}

    c = TuneCache(path)
    r1 = c.lookup_or_tune("k", tune)
    r2 = TuneCache(path).lookup_or_tune("k", tune)
    assert len(calls) == 1 and not r1["cached"] and r2["cached"]
    assert (r2["tile_bits"], r2["low_bits"]) == (13, 2)
