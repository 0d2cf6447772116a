"""Thin ctypes binding of libqsim.so (the C ABI in include/qsim.h).

Only argument marshalling lives here: every step of the simulation runs in the
CUDA library.  PyTorch supplies device memory (state buffers are torch tensors
the library views through qs_state_create's dev_buf) and the CUDA stream.  If
the library has not been built, every entry point raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import inputs as I

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libqsim.so")

C64, C128 = 0, 1
KIND = {"I": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8, "SWAP": 9,
        "RX": 16, "RY": 17, "RZ": 18, "PS": 19, "RXX": 20, "RYY": 21, "RZZ": 22, "MATRIX": 32}
STATUS = {0: "QS_OK", 1: "QS_ERR_INVALID_ARG", 2: "QS_ERR_OUT_OF_MEMORY", 3: "QS_ERR_CUDA",
          4: "QS_ERR_TIMEOUT", 5: "QS_ERR_UNSUPPORTED"}

# (name, argtypes) of every exported entry point, in header order.
_VP, _I, _D, _U64, _SZ = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_size_t
_PD = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int)
_PU64 = C.POINTER(C.c_uint64)
_PVP = C.POINTER(C.c_void_p)
SIGNATURES = [
    ("qs_version", []),
    ("qs_last_error", []),
    ("qs_state_create", [_I, _I, _VP, _SZ, _VP, _PVP]),
    ("qs_state_destroy", [_VP]),
    ("qs_state_device_ptr", [_VP, _PVP]),
    ("qs_state_set_basis", [_VP, _U64]),
    ("qs_state_set_plus", [_VP]),
    ("qs_state_copy_in", [_VP, _VP, _I]),
    ("qs_state_copy_out", [_VP, _VP, _I]),
    ("qs_state_copy", [_VP, _VP]),
    ("qs_state_norm2", [_VP, _PD]),
    ("qs_circuit_create", [_I, _PVP]),
    ("qs_circuit_destroy", [_VP]),
    ("qs_circuit_add", [_VP, _I, _PI, _I, _PI, _I, _I, _D, _D, _PD]),
    ("qs_circuit_finalize", [_VP, _I, _VP]),
    ("qs_circuit_codegen", [_VP, _VP, _I, _I, C.c_char_p, _SZ, C.POINTER(_SZ), _PI, C.POINTER(_SZ)]),
    ("qs_circuit_info", [_VP, _PI, _PI, _PI]),
    ("qs_apply_circuit", [_VP, _VP, _PD, _I]),
    ("qs_circuit_autotune", [_VP, _VP, _PD, _I, _I, _VP, _PD]),
    ("qs_dm_circuit_create", [_I, _PVP]),
    ("qs_dm_add_gate", [_VP, _I, _PI, _I, _PI, _I, _I, _D, _D, _PD]),
    ("qs_dm_add_channel", [_VP, _I, _I, _PD, _I, _PD]),
    ("qs_dm_expectation", [_VP, _VP, _PD]),
    ("qs_traj_create", [_I, _I, _VP, _PVP]),
    ("qs_traj_destroy", [_VP]),
    ("qs_traj_add_gate", [_VP, _I, _PI, _I, _PI, _I, _I, _D, _D]),
    ("qs_traj_add_channel", [_VP, _I, _I, _PD, _I, _PD]),
    ("qs_traj_info", [_VP, _PI, _PI, _PI, _PI]),
    ("qs_traj_run", [_VP, _VP, _PD, _I, _U64, C.c_longlong, _I, _PD, _PD, C.POINTER(C.c_ubyte)]),
    ("qs_traj_run_device", [_VP, _VP, _VP, _U64, C.c_longlong, _I, _VP, _VP]),
    ("qs_traj_state", [_VP, _PD, _I, _U64, C.c_longlong, _VP]),
    ("qs_apply_matrix", [_VP, _I, _PI, _PD, _I]),
    ("qs_ham_create", [_I, _I, _PU64, _PU64, _PD, _PVP]),
    ("qs_ham_destroy", [_VP]),
    ("qs_apply_hamiltonian", [_VP, _VP, _VP]),
    ("qs_expectation", [_VP, _VP, _PD]),
    ("qs_inner_product", [_VP, _VP, _PD]),
    ("qs_expectation_with_grad", [_VP, _VP, _VP, _VP, _PD, _I, _PD, _PD]),
    ("qs_sample", [_VP, _U64, _U64, _PU64]),
    ("qs_expectation_with_grad_multi", [_VP, _VP, _VP, _I, _VP, _PD, _I, _PD, _PD]),
    ("qs_expectation_general", [_VP, _VP, _VP, _VP, _VP, _VP, _PD, _I, _PD, _PD]),
    ("qs_measure", [_VP, _I, _U64, _PI]),
    ("qs_qaoa_create", [_I, _PI, _I, _I, _D, _I, _VP, _PVP]),
    ("qs_qaoa_destroy", [_VP]),
    ("qs_qaoa_info", [_VP, _PI, _PI, _PD]),
    ("qs_qaoa_max_cut", [_VP, _PI]),
    ("qs_qaoa_evolve", [_VP, _VP, _PD, _PD]),
    ("qs_qaoa_expectation", [_VP, _VP, _PD, _PD, _PD]),
    ("qs_qaoa_expectation_with_grad", [_VP, _VP, _VP, _PD, _PD, _PD, _PD, _PD]),
    ("qs_qaoa_xplan", [_I, _PI, _I, _I, _D, _I, _I, _I, C.POINTER(C.c_longlong), _I, _PI, _PI, _PD, _I, _PI]),
    ("qs_qaoa_xcoef", [_I, _PI, _I, _I, _D, _I, _I, _PD, _PD, _PD, _I, _PI, _PI]),
    ("qs_qaoa_evaluate", [_I, _PI, _I, _I, _D, _PD, _PD, _I, _PD, _PD, _PD]),
    ("qs_batch_create", [_I, _PI, _PI, _VP, _PI, _PU64, _PU64, _PD, _PI, _I, _VP, _PVP]),
    ("qs_batch_destroy", [_VP]),
    ("qs_batch_info", [_VP, _PI, _PI, _PI]),
    ("qs_batch_expectation_with_grad", [_VP, _PD, _PD, _PD]),
    ("qs_batch_expectation_with_grad_device", [_VP, _VP, _VP, _VP]),
    ("qs_graphs_create", [_I, _PI, _PI, _PI, _PVP]),
    ("qs_graphs_destroy", [_VP]),
    ("qs_gnn_n_weights", [_I, _I, _I, _PI]),
    ("qs_gnn_create", [_I, _I, _I, _VP, _PVP]),
    ("qs_gnn_destroy", [_VP]),
    ("qs_gnn_set_weights", [_VP, _VP, _I]),
    ("qs_gnn_get_weights", [_VP, _VP, _VP, _I]),
    ("qs_gnn_get_state", [_VP, _VP, _VP, _VP, _PI]),
    ("qs_gnn_set_state", [_VP, _VP, _VP, _VP, _I]),
    ("qs_gnn_forward", [_VP, _VP, _VP]),
    ("qs_gnn_backward", [_VP, _VP, _VP, _VP]),
    ("qs_gnn_adam_step", [_VP, _VP, C.c_float, C.c_float, C.c_float, C.c_float]),
    ("qs_gnn_train_step", [_VP, _VP, _VP, C.c_float, C.c_float, C.c_float, C.c_float, _VP]),
    ("qs_mse", [_I, _VP, _VP, _VP, _VP, _VP]),
    ("qs_adam_f64", [_I, _VP, _VP, _VP, _VP, _I, _D, _D, _D, _D, _I, _VP]),
    ("qs_expectation_noalloc", [_VP, _I, _I, _I, _PU64, _PU64, _PD, _VP, _PD]),
    ("qs_selftest_wait_timeout", [_PI]),
    ("qs_trace_enable", [_I]),
    ("qs_trace_read", [_I, _PI, _PD, _PD, _PI]),
]


class QSimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("fuse", C.c_int), ("tile_bits", C.c_int), ("low_bits", C.c_int), ("checkpoint", C.c_int)]


_lib = None


def lib():
    """Load libqsim.so (built by paper_2406_17248_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libqsim.so is not built ({LIB_PATH}); run paper_2406_17248_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name in ("qs_version", "qs_last_error") else C.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise QSimError(status, lib().qs_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


# --------------------------------------------------------------------------- states

class State:
    """A 2^n amplitude state in a torch-owned device buffer (complex64 / complex128)."""

    def __init__(self, n: int, dtype: int = C64, stream=None, device=None):
        import torch
        self.n, self.dtype = n, dtype
        ne = max(n, 4)
        tdt = torch.complex64 if dtype == C64 else torch.complex128
        self.buffer = torch.empty(1 << ne, dtype=tdt, device=device or "cuda")
        # the stream the library's state handle enqueues on (fixed at creation)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().qs_state_create(n, dtype, C.c_void_p(self.buffer.data_ptr()),
                                     self.buffer.numel() * self.buffer.element_size(),
                                     C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qs_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def amplitudes(self):
        """Zero-copy torch view of the 2^n amplitudes (device)."""
        return self.buffer[: 1 << self.n]

    def set_basis(self, index: int = 0):
        _check(lib().qs_state_set_basis(self.h, index))
        return self

    def set_plus(self):
        _check(lib().qs_state_set_plus(self.h))
        return self

    def set_qs(self, amps: np.ndarray):
        a = np.ascontiguousarray(amps, dtype=np.complex64 if self.dtype == C64 else np.complex128)
        if a.size != 1 << self.n:
            raise ValueError("wrong number of amplitudes")
        _check(lib().qs_state_copy_in(self.h, a.ctypes.data_as(C.c_void_p), 0))
        return self

    def get_qs(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex64 if self.dtype == C64 else np.complex128)
        _check(lib().qs_state_copy_out(self.h, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def copy_from(self, other: "State"):
        _check(lib().qs_state_copy(self.h, other.h))
        return self

    def norm2(self) -> float:
        v = C.c_double()
        _check(lib().qs_state_norm2(self.h, C.byref(v)))
        return v.value


# --------------------------------------------------------------------------- circuits

class Circuit:
    def __init__(self, n: int):
        self.n = n
        h = C.c_void_p()
        _check(lib().qs_circuit_create(n, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qs_circuit_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, kind: str, targets: Sequence[int], ctrls: Sequence[int] = (), param: int = -1,
            coef: float = 1.0, const: float = 0.0, matrix=None):
        t = (C.c_int * len(targets))(*targets)
        c = (C.c_int * max(len(ctrls), 1))(*ctrls) if ctrls else None
        m = None
        if matrix is not None:
            mm = np.asarray(matrix, dtype=np.complex128).reshape(-1)
            inter = np.empty(2 * mm.size)
            inter[0::2], inter[1::2] = mm.real, mm.imag
            self._keep = inter
            m = _dptr(inter)
        _check(lib().qs_circuit_add(self.h, KIND[kind], t, len(targets), c, len(ctrls), param, coef, const, m))
        return self

    def finalize(self, dtype: int = C64, fuse: int = 0, tile_bits: int = 0, low_bits: int = 0, checkpoint: int = 0):
        """checkpoint > 0: adjoint state checkpoints every `checkpoint` gates."""
        o = Options(fuse, tile_bits, low_bits, checkpoint)
        _check(lib().qs_circuit_finalize(self.h, dtype, C.byref(o)))
        return self

    def codegen(self, which: int = 0, compile: bool = False, tile_bits: int = 0, low_bits: int = 0,
                fuse: int = 4, cap: int = 1 << 22):
        """Source of the per-circuit micro-op kernels of the forward (which = 0) or
        adjoint (1) plan, compiled for sm_103a when `compile` (qs_circuit_codegen;
        host only, the circuit must not be finalized).  Returns {"source",
        "passes", "cubin_bytes"}."""
        o = Options(fuse, tile_bits, low_bits, 0)
        buf = C.create_string_buffer(cap)
        ln, ng, cb = C.c_size_t(), C.c_int(), C.c_size_t()
        _check(lib().qs_circuit_codegen(self.h, C.byref(o), which, int(bool(compile)), buf, cap, C.byref(ln),
                                        C.byref(ng), C.byref(cb)))
        if ln.value >= cap:
            raise RuntimeError(f"generated source of {ln.value} bytes does not fit {cap}")
        return {"source": buf.value.decode(), "passes": ng.value, "cubin_bytes": cb.value}

    def info(self):
        g, p, s = C.c_int(), C.c_int(), C.c_int()
        _check(lib().qs_circuit_info(self.h, C.byref(g), C.byref(p), C.byref(s)))
        return {"gates": g.value, "params": p.value, "passes": s.value}

    def apply(self, state: State, params=None):
        pr = np.ascontiguousarray(params if params is not None else np.zeros(0), dtype=np.float64)
        _check(lib().qs_apply_circuit(state.h, self.h, _dptr(pr) if pr.size else None, int(pr.size)))
        return state

    def autotune(self, state: State, params=None, reps: int = 2):
        """Pick the tile shape by timing (qs_circuit_autotune); overwrites `state`.
        Returns {"tile_bits", "low_bits", "ms"}."""
        pr = np.ascontiguousarray(params if params is not None else np.zeros(0), dtype=np.float64)
        o = Options(0, 0, 0, 0)
        ms = C.c_double()
        _check(lib().qs_circuit_autotune(self.h, state.h, _dptr(pr) if pr.size else None, int(pr.size), reps,
                                         C.byref(o), C.byref(ms)))
        return {"tile_bits": o.tile_bits, "low_bits": o.low_bits, "ms": ms.value}


def circuit_from(circ: I.Circuit) -> Circuit:
    c = Circuit(circ.n_qubits)
    for g in circ.gates:
        c.add(g.kind, g.targets, g.ctrls, g.param, g.coef, g.const,
              None if g.matrix is None else np.asarray(g.matrix))
    return c


class Hamiltonian:
    def __init__(self, ham: I.PauliSum):
        self.n = ham.n_qubits
        x = np.ascontiguousarray(ham.xmask, dtype=np.uint64)
        z = np.ascontiguousarray(ham.zmask, dtype=np.uint64)
        cf = np.ascontiguousarray(ham.coef, dtype=np.float64)
        h = C.c_void_p()
        _check(lib().qs_ham_create(self.n, int(cf.size), x.ctypes.data_as(_PU64), z.ctypes.data_as(_PU64),
                                   _dptr(cf), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qs_ham_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expectation(state: State, ham: Hamiltonian) -> float:
    v = C.c_double()
    _check(lib().qs_expectation(state.h, ham.h, C.byref(v)))
    return v.value


def apply_hamiltonian(dst: State, src: State, ham: Hamiltonian) -> State:
    _check(lib().qs_apply_hamiltonian(dst.h, src.h, ham.h))
    return dst


def inner_product(bra: State, ket: State) -> complex:
    out = np.zeros(2)
    _check(lib().qs_inner_product(bra.h, ket.h, _dptr(out)))
    return complex(out[0], out[1])


def expectation_with_grad(psi: State, lam: State, circ: Circuit, ham: Hamiltonian, params):
    pr = np.ascontiguousarray(params, dtype=np.float64)
    grad = np.zeros(max(pr.size, 1))
    e = C.c_double()
    _check(lib().qs_expectation_with_grad(psi.h, lam.h, circ.h, ham.h, _dptr(pr) if pr.size else None,
                                          int(pr.size), C.byref(e), _dptr(grad)))
    return e.value, grad[: pr.size]


def expectation_with_grad_multi(psi: State, lam: State, circ: Circuit, hams, params):
    """Energies [n_ham] and gradients [n_ham, n_params] for a list of Hamiltonians
    (one forward sweep, one reverse sweep per Hamiltonian)."""
    pr = np.ascontiguousarray(params, dtype=np.float64)
    n_ham = len(hams)
    arr = (C.c_void_p * n_ham)(*[h.h for h in hams])
    e = np.zeros(n_ham)
    g = np.zeros(max(n_ham * pr.size, 1))
    _check(lib().qs_expectation_with_grad_multi(psi.h, lam.h, circ.h, n_ham, C.cast(arr, C.c_void_p),
                                                _dptr(pr) if pr.size else None, int(pr.size), _dptr(e), _dptr(g)))
    return e, g[: n_ham * pr.size].reshape(n_ham, pr.size)


def expectation_general(psi: State, phi: State, lam: State, c_right: Circuit, c_left: Optional[Circuit],
                        ham: Hamiltonian, params):
    """E = <phi|U_l^dag H U_r|psi> and dE/dparams, both complex (qs_expectation_general);
    c_left None: U_l = U_r."""
    pr = np.ascontiguousarray(params, dtype=np.float64)
    e = np.zeros(2)
    g = np.zeros(2 * max(pr.size, 1))
    _check(lib().qs_expectation_general(psi.h, phi.h, lam.h, c_right.h, c_left.h if c_left is not None else None,
                                        ham.h, _dptr(pr) if pr.size else None, int(pr.size), _dptr(e), _dptr(g)))
    return complex(e[0], e[1]), g[: 2 * pr.size].view(np.complex128)


def measure(state: State, qubit: int, seed: int) -> int:
    """Measure one qubit (projective, in place); returns the outcome 0 or 1."""
    o = C.c_int()
    _check(lib().qs_measure(state.h, qubit, seed, C.byref(o)))
    return o.value


def sample(state: State, shots: int, seed: int) -> np.ndarray:
    out = np.zeros(max(shots, 1), dtype=np.uint64)
    _check(lib().qs_sample(state.h, shots, seed, out.ctypes.data_as(_PU64)))
    return out[:shots]


class BatchGate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_targets", C.c_int32), ("targets", C.c_int32 * 2),
                ("ctrl_mask", C.c_uint64), ("param", C.c_int32), ("pad", C.c_int32),
                ("coef", C.c_double), ("constant", C.c_double)]


# numpy twin of qs_batch_gate (same field order, sizes and offsets)
BATCH_GATE_DTYPE = np.dtype([("kind", "<i4"), ("n_targets", "<i4"), ("targets", "<i4", (2,)), ("ctrl_mask", "<u8"),
                             ("param", "<i4"), ("pad", "<i4"), ("coef", "<f8"), ("constant", "<f8")])
assert BATCH_GATE_DTYPE.itemsize == C.sizeof(BatchGate) == 48


class Batch:
    """Independent (circuit, Hamiltonian, parameters) instances evaluated in one
    persistent launch (qs_batch_*)."""

    def __init__(self, instances, dtype: int = C64, stream=None):
        n_inst = len(instances)
        nq = np.array([it.circuit.n_qubits for it in instances], dtype=np.int32)
        g_off, t_off, p_off = [0], [0], [0]
        rows, xs, zs, cs = [], [], [], []
        for it in instances:
            for g in it.circuit.gates:
                if g.kind == "MATRIX":
                    raise ValueError("MATRIX gates are not batched")
                t1 = g.targets[1] if len(g.targets) > 1 else g.targets[0]
                rows.append((KIND[g.kind], len(g.targets), (g.targets[0], t1), sum(1 << q for q in g.ctrls),
                             g.param, 0, g.coef, g.const))
            g_off.append(len(rows))
            xs.extend(int(v) for v in it.ham.xmask)
            zs.extend(int(v) for v in it.ham.zmask)
            cs.extend(float(v) for v in it.ham.coef)
            t_off.append(len(cs))
            p_off.append(p_off[-1] + it.circuit.n_params)
        self.n_inst, self.dtype = n_inst, dtype
        self.param_offsets = np.array(p_off, dtype=np.int32)
        gates = np.array(rows or [(0, 1, (0, 0), 0, -1, 0, 0.0, 0.0)], dtype=BATCH_GATE_DTYPE)
        x = np.array(xs or [0], dtype=np.uint64)
        z = np.array(zs or [0], dtype=np.uint64)
        cf = np.array(cs or [0.0], dtype=np.float64)
        go, to = np.array(g_off, dtype=np.int32), np.array(t_off, dtype=np.int32)
        h = C.c_void_p()
        _check(lib().qs_batch_create(n_inst, nq.ctypes.data_as(_PI), go.ctypes.data_as(_PI),
                                     gates.ctypes.data_as(C.c_void_p), to.ctypes.data_as(_PI),
                                     x.ctypes.data_as(_PU64), z.ctypes.data_as(_PU64), _dptr(cf),
                                     self.param_offsets.ctypes.data_as(_PI), dtype,
                                     C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(lib().qs_batch_info(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return {"instances": a.value, "params": b.value, "grid": c.value}

    def expectation_with_grad(self, params):
        """params: concatenated (instance order) or a list of per-instance arrays.
        Returns (energies[n_inst], list of per-instance gradient arrays)."""
        if isinstance(params, (list, tuple)):
            params = np.concatenate([np.asarray(p, dtype=np.float64) for p in params]) if params else np.zeros(0)
        pr = np.ascontiguousarray(params, dtype=np.float64)
        if pr.size != self.param_offsets[-1]:
            raise ValueError("wrong number of parameters")
        e = np.zeros(self.n_inst)
        g = np.zeros(max(pr.size, 1))
        _check(lib().qs_batch_expectation_with_grad(self.h, _dptr(pr) if pr.size else None, _dptr(e), _dptr(g)))
        po = self.param_offsets
        return e, [g[po[i]:po[i + 1]] for i in range(self.n_inst)]

    def expectation_with_grad_device(self, params, energies, grads):
        """Device (torch float64 CUDA tensor) variant: no copies, no synchronisation."""
        _check(lib().qs_batch_expectation_with_grad_device(self.h, C.c_void_p(params.data_ptr()),
                                                           C.c_void_p(energies.data_ptr()),
                                                           C.c_void_p(grads.data_ptr())))


CHANNELS = {"pauli": 0, "depolarizing": 1, "amplitude_damping": 2, "phase_damping": 3, "kraus": 4}


class DensityCircuit(Circuit):
    """A density-matrix circuit of n qubits (qs_dm_*): a 2n-qubit circuit holding
    each gate and its conjugate, and channels as superoperators."""

    def __init__(self, n: int):
        self.n_sys = n
        h = C.c_void_p()
        _check(lib().qs_dm_circuit_create(n, C.byref(h)))
        self.h = h

    def add(self, kind: str, targets: Sequence[int], ctrls: Sequence[int] = (), param: int = -1,
            coef: float = 1.0, const: float = 0.0, matrix=None):
        t = (C.c_int * len(targets))(*targets)
        cc = (C.c_int * max(len(ctrls), 1))(*ctrls) if ctrls else None
        m = None
        if matrix is not None:
            mm = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128)).view(np.float64).reshape(-1)
            m = mm.ctypes.data_as(_PD)
            self._keep = mm
        _check(lib().qs_dm_add_gate(self.h, KIND[kind], t, len(targets), cc, len(ctrls), param, coef, const, m))
        return self

    def add_channel(self, kind: str, qubit: int, p=(), kraus=None):
        pr = np.ascontiguousarray(p if len(p) else [0.0], dtype=np.float64)
        kr = None
        nk = 0
        if kraus is not None:
            ka = np.ascontiguousarray(np.asarray(kraus, dtype=np.complex128)).view(np.float64).reshape(-1)
            nk = len(kraus)
            kr = ka.ctypes.data_as(_PD)
            self._keep_k = ka
        _check(lib().qs_dm_add_channel(self.h, CHANNELS[kind], qubit, _dptr(pr), nk, kr))
        return self


def dm_circuit_from(circ: I.Circuit, channels_after=None) -> DensityCircuit:
    """Density-matrix circuit of an inputs.Circuit; channels_after[i] = [(kind, p,
    qubit)] added after gate i (key -1: before the first gate)."""
    ch = channels_after or {}
    c = DensityCircuit(circ.n_qubits)
    for kind, p, q in ch.get(-1, []):
        c.add_channel(kind, q, p)
    for i, g in enumerate(circ.gates):
        c.add(g.kind, g.targets, g.ctrls, g.param, g.coef, g.const,
              None if g.matrix is None else np.asarray(g.matrix).reshape(1 << len(g.targets), -1))
        for kind, p, q in ch.get(i, []):
            c.add_channel(kind, q, p)
    return c


class Trajectories:
    """Monte-Carlo trajectories of a noisy circuit (qs_traj_*; §3.3): each
    trajectory samples one branch per channel site; the mean of the trajectory
    energies estimates tr(rho H)."""

    def __init__(self, n: int, dtype: int = C64, stream=None):
        self.n, self.dtype = n, dtype
        h = C.c_void_p()
        _check(lib().qs_traj_create(n, dtype, C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qs_traj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, kind: str, targets: Sequence[int], ctrls: Sequence[int] = (), param: int = -1,
            coef: float = 1.0, const: float = 0.0):
        t = (C.c_int * len(targets))(*targets)
        cc = (C.c_int * max(len(ctrls), 1))(*ctrls) if ctrls else None
        _check(lib().qs_traj_add_gate(self.h, KIND[kind], t, len(targets), cc, len(ctrls), param, coef, const))
        return self

    def add_channel(self, kind: str, qubit: int, p=(), kraus=None):
        pr = np.ascontiguousarray(p if len(p) else [0.0], dtype=np.float64)
        kr, nk = None, 0
        if kraus is not None:
            ka = np.ascontiguousarray(np.asarray(kraus, dtype=np.complex128)).view(np.float64).reshape(-1)
            nk = len(kraus)
            kr = ka.ctypes.data_as(_PD)
            self._keep_k = ka
        _check(lib().qs_traj_add_channel(self.h, CHANNELS[kind], qubit, _dptr(pr), nk, kr))
        return self

    def info(self):
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().qs_traj_info(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return {"sites": a.value, "params": b.value, "grid_energy": c.value, "grid_grad": d.value}

    def run(self, ham: Hamiltonian, params, n_traj: int, seed: int, first: int = 0, grad: bool = False,
            choices: bool = False):
        """Energies [n_traj] (+ mean gradient [n_params]) (+ branches [n_traj, n_sites])."""
        pr = np.ascontiguousarray(params, dtype=np.float64)
        e = np.zeros(n_traj)
        g = np.zeros(max(pr.size, 1)) if grad else None
        ns = self.info()["sites"]
        ch = np.zeros((n_traj, max(ns, 1)), dtype=np.uint8) if choices else None
        _check(lib().qs_traj_run(self.h, ham.h, _dptr(pr) if pr.size else None, int(pr.size), seed, first, n_traj,
                                 _dptr(e), _dptr(g) if grad else None,
                                 ch.ctypes.data_as(C.POINTER(C.c_ubyte)) if choices else None))
        out = [e]
        if grad:
            out.append(g[: pr.size])
        if choices:
            out.append(ch[:, :ns])
        return out[0] if len(out) == 1 else tuple(out)

    def run_device(self, ham: Hamiltonian, params, n_traj: int, seed: int, energies, grad_mean=None, first: int = 0):
        """Device (torch float64 CUDA tensors) variant: no copies and no
        synchronisation while the state fits in shared memory (larger states
        run trajectory by trajectory and synchronise)."""
        _check(lib().qs_traj_run_device(self.h, ham.h, C.c_void_p(params.data_ptr()) if params.numel() else None,
                                        seed, first, n_traj, C.c_void_p(energies.data_ptr()),
                                        C.c_void_p(grad_mean.data_ptr()) if grad_mean is not None else None))

    def state(self, params, seed: int, traj: int, out: "State") -> "State":
        pr = np.ascontiguousarray(params, dtype=np.float64)
        _check(lib().qs_traj_state(self.h, _dptr(pr) if pr.size else None, int(pr.size), seed, traj, out.h))
        return out


def trajectories_from(circ: I.Circuit, channels_after=None, dtype: int = C64, stream=None) -> Trajectories:
    """Trajectory engine of an inputs.Circuit; channels_after[i] = [(kind, p, qubit)
    or ("kraus", (), qubit, matrices)] added after gate i (key -1: first)."""
    ch = channels_after or {}
    t = Trajectories(circ.n_qubits, dtype, stream)

    def site(c):
        t.add_channel(c[0], c[2], c[1], c[3] if len(c) > 3 else None)

    for c in ch.get(-1, []):
        site(c)
    for i, g in enumerate(circ.gates):
        if g.kind == "MATRIX":
            raise ValueError("MATRIX gates are not supported in trajectories")
        t.add(g.kind, g.targets, g.ctrls, g.param, g.coef, g.const)
        for c in ch.get(i, []):
            site(c)
    return t


def dm_expectation(rho: State, ham: Hamiltonian) -> float:
    """tr(rho H) of a density-matrix state (2n qubits) for an n-qubit Pauli sum."""
    e = C.c_double()
    _check(lib().qs_dm_expectation(rho.h, ham.h, C.byref(e)))
    return e.value


def apply_matrix(state: State, targets, matrix, engine: int = 0) -> State:
    """psi <- U psi for a dense 2^k x 2^k complex matrix on `targets` (qs_apply_matrix);
    engine 0 automatic, 1 CUDA cores, 2 tensor cores."""
    t = np.ascontiguousarray(targets, dtype=np.int32)
    U = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
    k = int(t.size)
    if U.shape != (1 << k, 1 << k):
        raise ValueError("matrix must be 2^k x 2^k")
    m = np.ascontiguousarray(U.view(np.float64).reshape(-1))
    _check(lib().qs_apply_matrix(state.h, k, t.ctypes.data_as(_PI), _dptr(m), engine))
    return state


XPLAN_REC = 131


def qaoa_xplan(n: int, edges, p: int, gamma_scale: float = 1.0, tile_bits: int = 0, low_bits: int = 0,
               which: int = 0):
    """The complex64 two-shape QAOA plan (qs_qaoa_xplan, host only): a list of
    pass records (dicts) and the slot table [(output, weight)]."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    maxp, maxs = 512, 4096
    rec = (C.c_longlong * (maxp * XPLAN_REC))()
    so = (C.c_int * maxs)()
    sw = (C.c_double * maxs)()
    npass, nslot = C.c_int(), C.c_int()
    _check(lib().qs_qaoa_xplan(n, e.ctypes.data_as(_PI), int(e.size // 2), p, gamma_scale, tile_bits, low_bits,
                               which, rec, maxp, C.byref(npass), so, sw, maxs, C.byref(nslot)))
    out = []
    for i in range(npass.value):
        r = rec[i * XPLAN_REC:(i + 1) * XPLAN_REC]
        d = dict(two=r[0], flags=r[1], S=r[2], n_phases=r[3], c1=r[4], c3=r[5], cd=r[6], slot=r[7:10],
                 m=r[10], c=r[11], phases=[])
        for ph in range(r[3]):
            q = r[12 + 7 * ph:12 + 7 * ph + 7]
            d["phases"].append(dict(m1=q[0], m3=q[1], diag=q[2], reg=list(q[3:7])))
        d["cw"] = r[130]
        d["maps"] = []
        for k in range(2):
            t = r[96 + 17 * k:96 + 17 * k + 17]
            d["maps"].append(dict(e=t[0], lb=t[1], a=list(t[2:7]), w=list(t[7:12]), box=list(t[12:17])))
        out.append(d)
    return out, [(so[i], sw[i]) for i in range(nslot.value)]


def qaoa_xcoef(n: int, edges, p: int, gamma, beta, gamma_scale: float = 1.0, tile_bits: int = 0, low_bits: int = 0):
    """The per-call coefficient table of the complex64 two-shape QAOA passes
    (qs_qaoa_xcoef, host only): complex entries and whether the energy plan
    leaves every qubit flipped."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    maxe = 1 << 16
    tab = np.zeros(2 * maxe)
    ne, fl = C.c_int(), C.c_int()
    _check(lib().qs_qaoa_xcoef(n, e.ctypes.data_as(_PI), int(e.size // 2), p, gamma_scale, tile_bits, low_bits,
                               _dptr(g), _dptr(b), _dptr(tab), maxe, C.byref(ne), C.byref(fl)))
    t = tab[:2 * ne.value]
    return t[0::2] + 1j * t[1::2], bool(fl.value)


def expectation_noalloc(state: State, ham: I.PauliSum, stream=None) -> float:
    """<psi|H|psi> through qs_expectation_noalloc: no device allocation by the
    library (its working memory is a fixed array inside the library), for callers
    whose device memory belongs to another allocator.  Runs on the state's own
    stream unless another is given, behind the state's pending work."""
    if stream is None:
        stream = state._stream
    x = np.ascontiguousarray(ham.xmask, dtype=np.uint64)
    z = np.ascontiguousarray(ham.zmask, dtype=np.uint64)
    cf = np.ascontiguousarray(ham.coef, dtype=np.float64)
    e = C.c_double()
    _check(lib().qs_expectation_noalloc(C.c_void_p(state.buffer.data_ptr()), state.n, state.dtype, int(cf.size),
                                        x.ctypes.data_as(_PU64), z.ctypes.data_as(_PU64), _dptr(cf),
                                        C.c_void_p(_stream_ptr(stream)), C.byref(e)))
    return e.value


def trace_enable(on: bool = True):
    """Record a CUDA event pair around every tile-pass launch (see qs_trace_enable)."""
    _check(lib().qs_trace_enable(1 if on else 0))


TRACE_KINDS = {0: "tile_pass_kernel", 1: "qaoa_pass_kernel (psi)", 2: "qaoa_pass_kernel (psi, lam)",
               3: "qaoa_il_kernel (interleaved reverse)", 4: "batch_kernel", 5: "dense_tc_kernel (tcgen05)",
               6: "dense_cc_kernel", 7: "qx_kernel<false> (psi, forward)", 8: "qx_kernel<true> (turnaround)",
               9: "qx_kernel<true> (psi/lam interleaved, reverse)", 10: "tile2_kernel (micro-op tile pass)",
               11: "qs_t2g (per-circuit micro-op tile pass)"}


def trace_read(max_records: int = 65536):
    """(durations in ms, algorithmic bytes, kernel kinds) of the recorded launches."""
    ms = np.zeros(max_records)
    by = np.zeros(max_records)
    kinds = np.zeros(max_records, dtype=np.int32)
    n = C.c_int()
    _check(lib().qs_trace_read(max_records, C.byref(n), _dptr(ms), _dptr(by), kinds.ctypes.data_as(_PI)))
    return ms[: n.value], by[: n.value], kinds[: n.value]


# --------------------------------------------------------------------------- QAOA

def qaoa_evaluate(n: int, edges, p: int, gamma, beta, gamma_scale: float = 1.0, dtype: int = C64):
    """One energy + gradient evaluation without handles (qs_qaoa_evaluate)."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    E = C.c_double()
    dg, db = np.zeros(p), np.zeros(p)
    _check(lib().qs_qaoa_evaluate(n, e.ctypes.data_as(_PI), int(e.size // 2), p, gamma_scale, _dptr(g), _dptr(b),
                                  dtype, C.byref(E), _dptr(dg), _dptr(db)))
    return E.value, dg, db


class QAOA:
    """MaxCut QAOA engine: |+>^n, p layers of exp(-i gs gamma C) then RX(beta)."""

    def __init__(self, n: int, edges, p: int, gamma_scale: float = 1.0, dtype: int = C64,
                 tile_bits: int = 0, low_bits: int = 0, checkpoint: int = 0, engine: int = 0):
        """checkpoint > 0: adjoint state checkpoints every `checkpoint` layers.
        engine: 0 automatic, 1 the general tile passes, 2 the complex64
        two-shape passes (tile_bits / low_bits then give the reverse tile)."""
        self.n, self.p, self.dtype = n, p, dtype
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
        self._edges = e
        o = Options(engine, tile_bits, low_bits, checkpoint)
        h = C.c_void_p()
        _check(lib().qs_qaoa_create(n, e.ctypes.data_as(_PI), int(e.size // 2), p, gamma_scale, dtype,
                                    C.byref(o), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qs_qaoa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        f, r, b = C.c_int(), C.c_int(), C.c_double()
        _check(lib().qs_qaoa_info(self.h, C.byref(f), C.byref(r), C.byref(b)))
        return {"fwd_passes": f.value, "rev_passes": r.value, "bytes_per_eval": b.value}

    def _angles(self, gamma, beta):
        g = np.ascontiguousarray(gamma, dtype=np.float64)
        b = np.ascontiguousarray(beta, dtype=np.float64)
        if g.size != self.p or b.size != self.p:
            raise ValueError("gamma and beta need p entries each")
        return g, b

    def evolve(self, psi: State, gamma, beta) -> State:
        g, b = self._angles(gamma, beta)
        _check(lib().qs_qaoa_evolve(self.h, psi.h, _dptr(g), _dptr(b)))
        return psi

    def expectation(self, psi: State, gamma, beta) -> float:
        g, b = self._angles(gamma, beta)
        e = C.c_double()
        _check(lib().qs_qaoa_expectation(self.h, psi.h, _dptr(g), _dptr(b), C.byref(e)))
        return e.value

    def expectation_with_grad(self, psi: State, lam: State, gamma, beta):
        g, b = self._angles(gamma, beta)
        e = C.c_double()
        dg, db = np.zeros(self.p), np.zeros(self.p)
        _check(lib().qs_qaoa_expectation_with_grad(self.h, psi.h, lam.h, _dptr(g), _dptr(b), C.byref(e),
                                                   _dptr(dg), _dptr(db)))
        return e.value, dg, db

    def max_cut(self) -> int:
        """MaxCut optimum by exhaustive search over the device cut-value array."""
        m = C.c_int()
        _check(lib().qs_qaoa_max_cut(self.h, C.byref(m)))
        return m.value


# --------------------------------------------------------------------------- learned initialiser (GNN)

def _dev(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class Graphs:
    """A validated device copy of a CSR batch of graphs (qs_graphs_create)."""

    def __init__(self, node_off, adj_off, adj):
        no = np.ascontiguousarray(node_off, dtype=np.int32)
        ao = np.ascontiguousarray(adj_off, dtype=np.int32)
        a = np.ascontiguousarray(adj, dtype=np.int32)
        if a.size == 0:
            a = np.zeros(1, dtype=np.int32)
        self.n_graphs = int(no.size - 1)
        h = C.c_void_p()
        _check(lib().qs_graphs_create(self.n_graphs, no.ctypes.data_as(_PI), ao.ctypes.data_as(_PI),
                                      a.ctypes.data_as(_PI), C.byref(h)))
        self.h = h

    @classmethod
    def from_graphs(cls, graphs):
        return cls(*I.pack_graphs(graphs))

    def close(self):
        if getattr(self, "h", None):
            lib().qs_graphs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gnn_n_weights(hidden: int = 64, layers: int = 3, out_dim: int = 8) -> int:
    n = C.c_int()
    _check(lib().qs_gnn_n_weights(hidden, layers, out_dim, C.byref(n)))
    return n.value


class GNN:
    """The graph network of qs_gnn_* (bfloat16 weights, float32 arithmetic)."""

    def __init__(self, hidden: int = 64, layers: int = 3, out_dim: int = 8, stream=None):
        self.hidden, self.layers, self.out_dim = hidden, layers, out_dim
        self.n_weights = gnn_n_weights(hidden, layers, out_dim)
        h = C.c_void_p()
        _check(lib().qs_gnn_create(hidden, layers, out_dim, C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qs_gnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, w):
        if isinstance(w, np.ndarray):
            a = np.ascontiguousarray(w, dtype=np.float32)
            if a.size != self.n_weights:
                raise ValueError("wrong number of weights")
            _check(lib().qs_gnn_set_weights(self.h, a.ctypes.data_as(C.c_void_p), 0))
        else:
            if w.numel() != self.n_weights:
                raise ValueError("wrong number of weights")
            _check(lib().qs_gnn_set_weights(self.h, _dev(w), 1))

    def save(self, path: str):
        """Checkpoint the training state (weights, Adam moments, step) to an .npz file."""
        w, m, v = (np.zeros(self.n_weights, dtype=np.float32) for _ in range(3))
        step = C.c_int()
        _check(lib().qs_gnn_get_state(self.h, w.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                      v.ctypes.data_as(C.c_void_p), C.byref(step)))
        np.savez(path, w=w, m=m, v=v, step=step.value,
                 dims=np.array([self.hidden, self.layers, self.out_dim], dtype=np.int64))

    def load(self, path: str):
        """Resume from a file written by save() (same dimensions)."""
        z = np.load(path)
        if tuple(int(x) for x in z["dims"]) != (self.hidden, self.layers, self.out_dim):
            raise ValueError("checkpoint dimensions differ from this network's")
        arrs = [np.ascontiguousarray(z[k], dtype=np.float32) for k in ("w", "m", "v")]
        _check(lib().qs_gnn_set_state(self.h, *(a.ctypes.data_as(C.c_void_p) for a in arrs), int(z["step"])))
        return self

    def get_weights(self):
        """(float32 master weights, bfloat16 bit patterns as uint16) on the host."""
        w = np.zeros(self.n_weights, dtype=np.float32)
        wb = np.zeros(self.n_weights, dtype=np.uint16)
        _check(lib().qs_gnn_get_weights(self.h, w.ctypes.data_as(C.c_void_p), wb.ctypes.data_as(C.c_void_p), 0))
        return w, wb

    def forward(self, graphs: Graphs, out):
        """out: device float32 tensor [n_graphs, out_dim] (written asynchronously)."""
        _check(lib().qs_gnn_forward(self.h, graphs.h, _dev(out)))
        return out

    def backward(self, graphs: Graphs, dout, grad):
        _check(lib().qs_gnn_backward(self.h, graphs.h, _dev(dout), _dev(grad)))
        return grad

    def adam_step(self, grad, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _check(lib().qs_gnn_adam_step(self.h, _dev(grad), lr, beta1, beta2, eps))

    def train_step(self, graphs: Graphs, targets, lr: float, loss=None, beta1: float = 0.9, beta2: float = 0.999,
                   eps: float = 1e-8):
        """Forward, MSE gradient, backward and Adam in two launches (qs_gnn_train_step)."""
        _check(lib().qs_gnn_train_step(self.h, graphs.h, _dev(targets), lr, beta1, beta2, eps,
                                       _dev(loss) if loss is not None else None))


def mse(y, target, loss=None, dy=None, stream=None):
    """Device float32 tensors: loss (1 element) and dy may be None."""
    _check(lib().qs_mse(int(y.numel()), _dev(y), _dev(target), _dev(loss) if loss is not None else None,
                        _dev(dy) if dy is not None else None, C.c_void_p(_stream_ptr(stream))))


def adam_f64(w, m, v, grad, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             maximize: bool = False, stream=None):
    """One in-place Adam step on device float64 tensors."""
    _check(lib().qs_adam_f64(int(w.numel()), _dev(w), _dev(m), _dev(v), _dev(grad), t, lr, beta1, beta2, eps,
                             1 if maximize else 0, C.c_void_p(_stream_ptr(stream))))
