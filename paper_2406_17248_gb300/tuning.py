"""Autotuner cache: the tile shape `qs_circuit_autotune` picks for a circuit,
kept in a JSON file keyed by GPU name, dtype, qubit count and the circuit's gate
structure (kinds, targets, controls -- not the angles), so a structure timed
once is finalised from the file afterwards.  Host bookkeeping only: the timing
itself is the library's."""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Dict, Optional

from . import inputs as I


def structure_key(circ: I.Circuit, dtype: int, gpu: str) -> str:
    h = hashlib.sha256()
    for g in circ.gates:
        h.update(repr((g.kind, tuple(g.targets), tuple(g.ctrls))).encode())
    return f"{gpu}|dtype={dtype}|n={circ.n_qubits}|gates={len(circ.gates)}|{h.hexdigest()[:16]}"


class TuneCache:
    """A JSON file mapping structure keys to {"tile_bits", "low_bits", "ms"}."""

    def __init__(self, path: str):
        self.path = path
        self.entries: Dict[str, dict] = {}
        if os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get(self, key: str) -> Optional[dict]:
        return self.entries.get(key)

    def put(self, key: str, value: dict):
        self.entries[key] = {k: value[k] for k in ("tile_bits", "low_bits", "ms")}
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def lookup_or_tune(self, key: str, tune: Callable[[], dict]) -> dict:
        """The cached choice, or tune() (which times and returns a choice) stored."""
        hit = self.get(key)
        if hit is not None:
            return dict(hit, cached=True)
        r = tune()
        self.put(key, r)
        return dict(r, cached=False)


def finalize_tuned(circ: I.Circuit, dtype: int, state, params, cache_path: str, reps: int = 2):
    """A finalised qsim.Circuit for `circ` with the tile shape from the cache, or
    picked by qs_circuit_autotune on `state` (overwritten) and then cached."""
    import torch
    from . import qsim as Q
    c = Q.circuit_from(circ)
    key = structure_key(circ, dtype, torch.cuda.get_device_name())
    choice = TuneCache(cache_path).lookup_or_tune(
        key, lambda: c.finalize(dtype).autotune(state, params, reps))
    if choice["cached"]:
        c.finalize(dtype, tile_bits=choice["tile_bits"], low_bits=choice["low_bits"])
    return c, choice
