"""FP64 CPU oracle for mixed-radix state-vector simulation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product library
never does.  It shares no code with the CUDA path (``oracle.c`` is plain C
compiled with gcc, loaded through ctypes).

The arithmetic lives in ``oracle.c``; this module only builds it, marshals
numpy arrays and loops over a circuit's gates in order (the circuit loop of
the paper's experiments: gates executed one after another).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.or_apply.restype = ctypes.c_int
        lib.or_apply.argtypes = [ctypes.c_int32, _i32p, _f64p, _f64p, ctypes.c_int32, _i32p,
                                 _f64p, ctypes.c_int32, _i32p, _i32p, ctypes.c_int32]
        lib.or_norm.restype = ctypes.c_double
        lib.or_norm.argtypes = [ctypes.c_int64, _f64p]
        lib.or_probabilities.restype = None
        lib.or_probabilities.argtypes = [ctypes.c_int64, _f64p, _f64p]
        lib.or_marginal.restype = ctypes.c_int
        lib.or_marginal.argtypes = [ctypes.c_int32, _i32p, _f64p, ctypes.c_int32, _f64p]
        lib.or_dim.restype = ctypes.c_int64
        lib.or_dim.argtypes = [ctypes.c_int32, _i32p]
        lib.or_max_threads.restype = ctypes.c_int32
        lib.or_max_threads.argtypes = []
        _lib = lib
        return lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def max_threads() -> int:
    return int(_load().or_max_threads())


def zero_state(dims) -> np.ndarray:
    """``|0...0>`` as a complex128 vector."""
    D = int(np.prod(np.asarray(dims, dtype=np.int64)))
    psi = np.zeros(D, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_gate(dims, psi: np.ndarray, gate, nthreads: int = 1,
               out: Optional[np.ndarray] = None) -> np.ndarray:
    """Return ``G psi`` for one gate (see ``oracle.c`` for the definition)."""
    lib = _load()
    dims_a = _i32(dims)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    if out is None:
        out = np.empty_like(psi)
    wires = _i32(gate.wires)
    cw = _i32(gate.controls if len(gate.controls) else [0])
    cv = _i32(gate.values if len(gate.values) else [0])
    U = np.ascontiguousarray(gate.U, dtype=np.complex128)
    rc = lib.or_apply(len(dims_a), _ptr(dims_a, _i32p), _ptr(psi.view(np.float64), _f64p),
                      _ptr(out.view(np.float64), _f64p), len(wires), _ptr(wires, _i32p),
                      _ptr(U.view(np.float64), _f64p), len(gate.controls), _ptr(cw, _i32p),
                      _ptr(cv, _i32p), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle rejected gate {gate.name} wires={gate.wires} "
                         f"controls={gate.controls} values={gate.values} (code {rc})")
    return out


def run_circuit(circ, psi0: Optional[np.ndarray] = None, nthreads: int = 1,
                max_gates: Optional[int] = None) -> np.ndarray:
    """Apply the circuit's gates in order to ``psi0`` (default ``|0...0>``)."""
    psi = zero_state(circ.dims) if psi0 is None else np.array(psi0, dtype=np.complex128)
    tmp = np.empty_like(psi)
    gates = circ.gates if max_gates is None else circ.gates[:max_gates]
    for g in gates:
        apply_gate(circ.dims, psi, g, nthreads=nthreads, out=tmp)
        psi, tmp = tmp, psi
    return psi


class _Gate:
    """Plain gate record (what :func:`apply_gate` reads), picklable."""

    def __init__(self, wires, U, controls, values, name):
        self.wires, self.U, self.controls, self.values, self.name = wires, U, controls, values, name


class _Circuit:
    def __init__(self, dims, gates):
        self.dims, self.gates = dims, gates


def _plain(circ) -> _Circuit:
    return _Circuit(tuple(int(d) for d in circ.dims),
                    [_Gate(tuple(g.wires), np.asarray(g.U), tuple(g.controls), tuple(g.values),
                           getattr(g, "name", "U")) for g in circ.gates])


def _run_one(circ) -> np.ndarray:
    return run_circuit(circ, nthreads=1)


def run_circuits(circs, workers: Optional[int] = None) -> list:
    """:func:`run_circuit` on many circuits, one single-threaded oracle per
    circuit in a pool of ``workers`` processes (default: all host cores).
    The pool is started with ``spawn``, so it is safe to use from a process
    that already holds a CUDA context."""
    import concurrent.futures as cf
    import multiprocessing as mp

    circs = [_plain(c) for c in circs]  # only what the oracle reads crosses the process boundary
    workers = workers or max(1, os.cpu_count() or 1)
    if workers == 1 or len(circs) <= 1:
        return [_run_one(c) for c in circs]
    build()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_run_one, circs, chunksize=max(1, len(circs) // (8 * workers))))


def norm(psi: np.ndarray) -> float:
    """Squared norm ``sum |psi_j|^2`` (compensated summation)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(_load().or_norm(psi.size, _ptr(psi.view(np.float64), _f64p)))


def probabilities(psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty(psi.size, dtype=np.float64)
    _load().or_probabilities(psi.size, _ptr(psi.view(np.float64), _f64p), _ptr(out, _f64p))
    return out


def marginal(dims, psi: np.ndarray, wire: int) -> np.ndarray:
    dims_a = _i32(dims)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty(int(dims_a[wire]), dtype=np.float64)
    rc = _load().or_marginal(len(dims_a), _ptr(dims_a, _i32p), _ptr(psi.view(np.float64), _f64p),
                             int(wire), _ptr(out, _f64p))
    if rc != 0:
        raise ValueError(f"oracle rejected marginal of wire {wire} (code {rc})")
    return out


def dim(dims) -> int:
    dims_a = _i32(dims)
    return int(_load().or_dim(len(dims_a), _ptr(dims_a, _i32p)))
