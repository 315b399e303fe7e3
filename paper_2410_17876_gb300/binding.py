"""ctypes binding of ``libqudit.so`` (C ABI in ``include/qudit.h``).

Argument marshalling only: every step of a gate application, readout or
reset runs in the library's CUDA kernels.  The module raises on import if
the library has not been built -- there is no CPU fallback.  PyTorch is used
for device memory (``State`` wraps a torch tensor) and streams.

The ``qd_*`` functions keep the C names and raise :class:`QuditError` on a
non-zero status instead of returning it.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

QD_OK, QD_ERR_ARG, QD_ERR_OOM, QD_ERR_CUDA, QD_ERR_TIMEOUT, QD_ERR_UNSUPPORTED, QD_ERR_DEVICE = range(7)
QD_C64, QD_C128 = 0, 1
QD_MAX_WIRES, QD_MAX_DIM, QD_MAX_GATE_DIM, QD_MAX_CONTROLS = 48, 64, 64, 16

# QD_BOUNDS=1 in the environment selects the bounds-checked build of the
# library (built by build.build(bounds=True) into its own directory).
LIB_PATH = _build.LIB_BOUNDS if os.environ.get("QD_BOUNDS") == "1" else _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqudit.so is not built ({LIB_PATH}); run paper_2410_17876_gb300.build.build() "
                      "or __graft_entry__.build() first -- there is no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class qd_plan_info(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("kind", ctypes.c_int32), ("vec", ctypes.c_int32),
                ("touched_rows", ctypes.c_int32), ("classes", ctypes.c_int64), ("run", ctypes.c_int64)]


QD_MAX_GATE_WIRES = 6
QD_FUSE_OFF, QD_FUSE_TILE, QD_FUSE_BLOCK = 0, 1, 2
QD_TC_TF32X3, QD_TC_BF16X3, QD_TC_OFF = 0, 1, 2
TC_MODES = {"tf32x3": QD_TC_TF32X3, "bf16x3": QD_TC_BF16X3, "fp32": QD_TC_OFF}


class qd_gate_desc(ctypes.Structure):
    _fields_ = [("n_wires", ctypes.c_int32), ("n_ctrl", ctypes.c_int32),
                ("wires", ctypes.c_int32 * QD_MAX_GATE_WIRES),
                ("ctrl_wires", ctypes.c_int32 * QD_MAX_CONTROLS),
                ("ctrl_vals", ctypes.c_int32 * QD_MAX_CONTROLS), ("matrix_offset", ctypes.c_int64)]


class qd_fusion_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("max_tile_amps", ctypes.c_int32), ("min_gates", ctypes.c_int32),
                ("min_row", ctypes.c_int32), ("block_dim", ctypes.c_int32), ("tc_mode", ctypes.c_int32)]


class qd_circuit(ctypes.Structure):
    _fields_ = [("n_wires", ctypes.c_int32), ("dims", ctypes.POINTER(ctypes.c_int32)), ("n_gates", ctypes.c_int32),
                ("gates", ctypes.POINTER(qd_gate_desc)), ("matrices", ctypes.POINTER(ctypes.c_double))]


class qd_batch_opts(ctypes.Structure):
    _fields_ = [("small_max_amps", ctypes.c_int32), ("n_streams", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("path", ctypes.c_int32), ("fusion", qd_fusion_opts)]


class qd_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("small_max_amps", ctypes.c_int32), ("max_group", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("fusion", qd_fusion_opts)]


class qd_request_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("kept", ctypes.c_int32),
                ("num_amplitudes", ctypes.c_int64), ("norm", ctypes.c_double), ("t_arrival", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


_SIGS = {
    "qd_state_create": (ctypes.c_int32, [_i32p, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.POINTER(_vp)]),
    "qd_state_wrap": (ctypes.c_int32, [_vp, ctypes.c_size_t, _i32p, ctypes.c_int32, ctypes.c_int32, _vp,
                                       ctypes.POINTER(_vp)]),
    "qd_state_destroy": (ctypes.c_int32, [_vp]),
    "qd_state_reset": (ctypes.c_int32, [_vp]),
    "qd_state_set_stream": (ctypes.c_int32, [_vp, _vp]),
    "qd_state_info": (ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int64), _i32p, _i32p]),
    "qd_state_device_ptr": (ctypes.c_int32, [_vp, ctypes.POINTER(_vp)]),
    "qd_state_set_amplitudes": (ctypes.c_int32, [_vp, _f64p]),
    "qd_state_get_amplitudes": (ctypes.c_int32, [_vp, _f64p]),
    "qd_state_get_raw": (ctypes.c_int32, [_vp, _vp, ctypes.c_size_t]),
    "qd_state_get_raw_async": (ctypes.c_int32, [_vp, _vp, ctypes.c_size_t]),
    "qd_apply_gate": (ctypes.c_int32, [_vp, ctypes.c_int32, _f64p]),
    "qd_apply_controlled": (ctypes.c_int32, [_vp, ctypes.c_int32, _f64p, _i32p, _i32p, ctypes.c_int32]),
    "qd_apply_multi": (ctypes.c_int32, [_vp, _i32p, ctypes.c_int32, _f64p, _i32p, _i32p, ctypes.c_int32]),
    "qd_norm": (ctypes.c_int32, [_vp, _f64p]),
    "qd_probabilities": (ctypes.c_int32, [_vp, _f64p]),
    "qd_probabilities_device": (ctypes.c_int32, [_vp, _vp]),
    "qd_marginal": (ctypes.c_int32, [_vp, ctypes.c_int32, _f64p]),
    "qd_synchronize": (ctypes.c_int32, [_vp]),
    "qd_set_fusion": (ctypes.c_int32, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "qd_set_lazy": (ctypes.c_int32, [_vp, ctypes.c_int32]),
    "qd_sparse_create": (ctypes.c_int32, [_i32p, ctypes.c_int32, _vp, ctypes.POINTER(_vp)]),
    "qd_sparse_destroy": (ctypes.c_int32, [_vp]),
    "qd_sparse_run": (ctypes.c_int32, [_vp, ctypes.POINTER(qd_gate_desc), ctypes.c_int32, _f64p]),
    "qd_sparse_nnz": (ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "qd_sparse_reserve": (ctypes.c_int32, [_vp, ctypes.c_int64]),
    "qd_sparse_get": (ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _f64p,
                                       ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "qd_apply_controlled_scan": (ctypes.c_int32, [_vp, ctypes.c_int32, _f64p, _i32p, _i32p, ctypes.c_int32]),
    "qd_flush": (ctypes.c_int32, [_vp]),
    "qd_norm_noalloc": (ctypes.c_int32, [_vp, ctypes.c_int64, ctypes.c_int32, _vp, _vp]),
    "qd_last_error": (ctypes.c_char_p, []),
    "qd_launch_count": (ctypes.c_uint64, []),
    "qd_bytes_uploaded": (ctypes.c_uint64, []),
    "qd_version": (ctypes.c_char_p, []),
    "qd_plan_gate": (ctypes.c_int32, [_i32p, ctypes.c_int32, ctypes.c_int32, _i32p, ctypes.c_int32, _f64p,
                                      _i32p, _i32p, ctypes.c_int32, ctypes.POINTER(qd_plan_info)]),
    "qd_selftest_host": (ctypes.c_int32, [ctypes.c_int32]),
    "qd_test_set_tc_wait": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_int32]),
    "qd_test_tc_ring_launches": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_int64)]),
    "qd_state_wire_to_top": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "qd_state_save": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_char_p]),
    "qd_bounds_status": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "qd_test_set_bounds_shrink": (ctypes.c_int32, [ctypes.c_int64]),
    "qd_state_load": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_char_p]),
    "qd_state_wire_from_top": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "qd_batch_create": (ctypes.c_int32, [ctypes.c_int32, _vp, ctypes.POINTER(_vp)]),
    "qd_batch_run": (ctypes.c_int32, [_vp, ctypes.POINTER(qd_circuit), ctypes.c_int32, ctypes.POINTER(qd_batch_opts)]),
    "qd_batch_relaunch": (ctypes.c_int32, [_vp]),
    "qd_batch_state": (ctypes.c_int32, [_vp, ctypes.c_int32, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int64)]),
    "qd_batch_get_amplitudes": (ctypes.c_int32, [_vp, ctypes.c_int32, _f64p]),
    "qd_batch_norms": (ctypes.c_int32, [_vp, _f64p]),
    "qd_batch_synchronize": (ctypes.c_int32, [_vp]),
    "qd_batch_destroy": (ctypes.c_int32, [_vp]),
    "qd_server_create": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(qd_server_opts), ctypes.POINTER(_vp)]),
    "qd_server_submit": (ctypes.c_int32, [_vp, ctypes.POINTER(qd_circuit), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "qd_server_submit_at": (ctypes.c_int32, [_vp, ctypes.POINTER(qd_circuit), ctypes.c_int32, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_uint64)]),
    "qd_server_poll": (ctypes.c_int32, [_vp, ctypes.POINTER(qd_request_result), ctypes.c_int32, _i32p]),
    "qd_server_drain": (ctypes.c_int32, [_vp, ctypes.c_double]),
    "qd_server_now": (ctypes.c_int32, [_vp, _f64p]),
    "qd_server_get_amplitudes": (ctypes.c_int32, [_vp, ctypes.c_uint64, _f64p]),
    "qd_server_release": (ctypes.c_int32, [_vp, ctypes.c_uint64]),
    "qd_server_destroy": (ctypes.c_int32, [_vp]),
    "qd_apply_circuit": (ctypes.c_int32, [_vp, ctypes.POINTER(qd_gate_desc), ctypes.c_int32, _f64p,
                                          ctypes.POINTER(qd_fusion_opts)]),
    "qd_plan_circuit": (ctypes.c_int32, [_i32p, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(qd_gate_desc),
                                         ctypes.c_int32, _f64p, ctypes.POINTER(qd_fusion_opts), _i32p, _i32p,
                                         ctypes.POINTER(ctypes.c_int64), _f64p, _i32p]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class QuditError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.qd_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {status}: {msg}")


def _check(rc: int, where: str) -> None:
    if rc != QD_OK:
        raise QuditError(rc, where)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def _mat(U) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(U, dtype=np.complex128)).view(np.float64)


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _opt_i32(a):
    if a is None or len(a) == 0:
        return None, np.zeros(1, np.int32)
    arr = _i32(a)
    return _p(arr, _i32p), arr


# --- C-ABI functions, same names ---------------------------------------------------------------
def qd_state_create(dims: Sequence[int], prec: int = QD_C128, stream: int = 0) -> int:
    d = _i32(dims)
    out = _vp()
    _check(_lib.qd_state_create(_p(d, _i32p), len(d), prec, _vp(stream), ctypes.byref(out)), "qd_state_create")
    return out.value


def qd_state_wrap(dev_ptr: int, nbytes: int, dims: Sequence[int], prec: int, stream: int = 0) -> int:
    d = _i32(dims)
    out = _vp()
    _check(_lib.qd_state_wrap(_vp(dev_ptr), nbytes, _p(d, _i32p), len(d), prec, _vp(stream), ctypes.byref(out)),
           "qd_state_wrap")
    return out.value


def qd_state_destroy(st: int) -> None:
    _check(_lib.qd_state_destroy(_vp(st)), "qd_state_destroy")


def qd_state_reset(st: int) -> None:
    _check(_lib.qd_state_reset(_vp(st)), "qd_state_reset")


def qd_state_set_stream(st: int, stream: int) -> None:
    _check(_lib.qd_state_set_stream(_vp(st), _vp(stream)), "qd_state_set_stream")


def qd_state_info(st: int):
    D = ctypes.c_int64()
    n = ctypes.c_int32()
    p = ctypes.c_int32()
    _check(_lib.qd_state_info(_vp(st), ctypes.byref(D), ctypes.byref(n), ctypes.byref(p)), "qd_state_info")
    return D.value, n.value, p.value


def qd_state_device_ptr(st: int) -> int:
    out = _vp()
    _check(_lib.qd_state_device_ptr(_vp(st), ctypes.byref(out)), "qd_state_device_ptr")
    return out.value


def qd_state_set_amplitudes(st: int, psi: np.ndarray) -> None:
    a = np.ascontiguousarray(psi, dtype=np.complex128).view(np.float64)
    D, _, _ = qd_state_info(st)
    if a.size != 2 * D:
        raise ValueError(f"expected {D} amplitudes, got {a.size // 2}")
    _check(_lib.qd_state_set_amplitudes(_vp(st), _p(a, _f64p)), "qd_state_set_amplitudes")


def qd_state_get_amplitudes(st: int) -> np.ndarray:
    D, _, _ = qd_state_info(st)
    out = np.empty(D, dtype=np.complex128)
    _check(_lib.qd_state_get_amplitudes(_vp(st), _p(out.view(np.float64), _f64p)), "qd_state_get_amplitudes")
    return out


def qd_state_get_raw(st: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    """Native-precision amplitudes (complex64 or complex128), no widening."""
    D, _, prec = qd_state_info(st)
    dt = np.complex64 if prec == QD_C64 else np.complex128
    if out is None:
        out = np.empty(D, dtype=dt)
    _check(_lib.qd_state_get_raw(_vp(st), _vp(out.ctypes.data), out.nbytes), "qd_state_get_raw")
    return out


def qd_state_get_raw_async(st: int, out: np.ndarray) -> np.ndarray:
    """Enqueue the copy of the native-precision amplitudes into ``out`` (a
    contiguous array the caller keeps alive, ideally page-locked) on the
    state's stream; read it after ``qd_synchronize``."""
    if not out.flags.c_contiguous:
        raise ValueError("out must be contiguous")
    _check(_lib.qd_state_get_raw_async(_vp(st), _vp(out.ctypes.data), out.nbytes), "qd_state_get_raw_async")
    return out


def qd_bounds_status():
    """(status, first_bad_index, checks_compiled) of the bounds-checked build's record (read and cleared)."""
    bad = ctypes.c_int64()
    comp = ctypes.c_int32()
    rc = _lib.qd_bounds_status(ctypes.byref(bad), ctypes.byref(comp))
    return int(rc), int(bad.value), int(comp.value)


def qd_test_set_bounds_shrink(amplitudes: int) -> None:
    _check(_lib.qd_test_set_bounds_shrink(int(amplitudes)), "qd_test_set_bounds_shrink")


def qd_state_save(st: int, path: str) -> None:
    _check(_lib.qd_state_save(_vp(st), str(path).encode()), "qd_state_save")


def qd_state_load(st: int, path: str) -> None:
    _check(_lib.qd_state_load(_vp(st), str(path).encode()), "qd_state_load")


def qd_state_wire_to_top(st: int, wire: int, dev_out: int) -> None:
    _check(_lib.qd_state_wire_to_top(_vp(st), int(wire), ctypes.c_void_p(dev_out)), "qd_state_wire_to_top")


def qd_state_wire_from_top(st: int, wire: int, dev_in: int) -> None:
    _check(_lib.qd_state_wire_from_top(_vp(st), int(wire), ctypes.c_void_p(dev_in)), "qd_state_wire_from_top")


def qd_apply_gate(st: int, target: int, U) -> None:
    _check(_lib.qd_apply_gate(_vp(st), int(target), _p(_mat(U), _f64p)), "qd_apply_gate")


def qd_apply_controlled(st: int, target: int, U, ctrl_wires, ctrl_vals) -> None:
    cw, cwa = _opt_i32(ctrl_wires)
    cv, cva = _opt_i32(ctrl_vals)
    n = 0 if ctrl_wires is None else len(ctrl_wires)
    _check(_lib.qd_apply_controlled(_vp(st), int(target), _p(_mat(U), _f64p), cw, cv, n), "qd_apply_controlled")


def qd_apply_controlled_scan(st: int, target: int, U, ctrl_wires, ctrl_vals) -> None:
    """The paper's scanning formulation of a controlled gate (every target class visited,
    its control digits tested), for comparison with ``qd_apply_controlled``."""
    cw, cwa = _opt_i32(ctrl_wires)
    cv, cva = _opt_i32(ctrl_vals)
    n = 0 if ctrl_wires is None else len(ctrl_wires)
    _check(_lib.qd_apply_controlled_scan(_vp(st), int(target), _p(_mat(U), _f64p), cw, cv, n),
           "qd_apply_controlled_scan")


def qd_apply_multi(st: int, wires, U, ctrl_wires=None, ctrl_vals=None) -> None:
    w = _i32(wires)
    cw, cwa = _opt_i32(ctrl_wires)
    cv, cva = _opt_i32(ctrl_vals)
    n = 0 if ctrl_wires is None else len(ctrl_wires)
    _check(_lib.qd_apply_multi(_vp(st), _p(w, _i32p), len(w), _p(_mat(U), _f64p), cw, cv, n), "qd_apply_multi")


def qd_norm(st: int) -> float:
    out = ctypes.c_double()
    _check(_lib.qd_norm(_vp(st), ctypes.byref(out)), "qd_norm")
    return out.value


def qd_probabilities(st: int) -> np.ndarray:
    D, _, _ = qd_state_info(st)
    out = np.empty(D, dtype=np.float64)
    _check(_lib.qd_probabilities(_vp(st), _p(out, _f64p)), "qd_probabilities")
    return out


def qd_probabilities_device(st: int, dev_out: int) -> None:
    _check(_lib.qd_probabilities_device(_vp(st), _vp(dev_out)), "qd_probabilities_device")


def qd_marginal(st: int, wire: int, d: int) -> np.ndarray:
    out = np.empty(int(d), dtype=np.float64)
    _check(_lib.qd_marginal(_vp(st), int(wire), _p(out, _f64p)), "qd_marginal")
    return out


def qd_synchronize(st: int) -> None:
    _check(_lib.qd_synchronize(_vp(st)), "qd_synchronize")


def qd_norm_noalloc(dev_amps: int, num_amplitudes: int, prec: int, stream: int, dev_out: int) -> None:
    """Squared norm of caller-owned device amplitudes into the device double at
    ``dev_out``, allocating nothing (for callers that cannot allocate, such as
    code under CUDA-graph capture); asynchronous on ``stream``."""
    _check(_lib.qd_norm_noalloc(_vp(dev_amps), int(num_amplitudes), int(prec), _vp(stream), _vp(dev_out)),
           "qd_norm_noalloc")


def qd_last_error() -> str:
    return _lib.qd_last_error().decode(errors="replace")


def qd_launch_count() -> int:
    return int(_lib.qd_launch_count())


def qd_bytes_uploaded() -> int:
    return int(_lib.qd_bytes_uploaded())


def qd_version() -> str:
    return _lib.qd_version().decode()


def qd_plan_gate(dims, prec, wires, U, ctrl_wires=None, ctrl_vals=None) -> dict:
    d = _i32(dims)
    w = _i32(wires)
    cw, cwa = _opt_i32(ctrl_wires)
    cv, cva = _opt_i32(ctrl_vals)
    n = 0 if ctrl_wires is None else len(ctrl_wires)
    info = qd_plan_info()
    _check(_lib.qd_plan_gate(_p(d, _i32p), len(d), prec, _p(w, _i32p), len(w), _p(_mat(U), _f64p), cw, cv, n,
                             ctypes.byref(info)), "qd_plan_gate")
    return {f: getattr(info, f) for f, _ in qd_plan_info._fields_}


def qd_test_set_tc_wait(spin_limit: int = 0, stall_producers: bool = False) -> None:
    """Testing hook: polls per bounded wait of the tensor-core block kernel (0 = default)
    and whether its producers publish nothing (so that its waits run out)."""
    _check(_lib.qd_test_set_tc_wait(int(spin_limit), 1 if stall_producers else 0), "qd_test_set_tc_wait")


def qd_test_tc_ring_launches() -> int:
    """Launches of the BF16x3 tile-ring kernel since the library was loaded."""
    out = ctypes.c_int64(0)
    _check(_lib.qd_test_tc_ring_launches(ctypes.byref(out)), "qd_test_tc_ring_launches")
    return int(out.value)


def qd_selftest_host(trials: int = 200) -> None:
    _check(_lib.qd_selftest_host(int(trials)), "qd_selftest_host")


_DESC_DTYPE = np.dtype([("n_wires", np.int32), ("n_ctrl", np.int32), ("wires", np.int32, QD_MAX_GATE_WIRES),
                        ("ctrl_wires", np.int32, QD_MAX_CONTROLS), ("ctrl_vals", np.int32, QD_MAX_CONTROLS),
                        ("matrix_offset", np.int64)], align=True)
assert _DESC_DTYPE.itemsize == ctypes.sizeof(qd_gate_desc)


def circuit_arrays(circuit):
    """(qd_gate_desc array, concatenated matrices) for a circuit; cached on the circuit object.

    The descriptors are a numpy structured array with the C layout of
    qd_gate_desc, so building them is a handful of vectorised assignments.
    """
    cache = getattr(circuit, "_qd_arrays", None)
    if cache is not None and cache[0] == len(circuit.gates):
        return cache[1], cache[2]
    gates = circuit.gates
    n = len(gates)
    d = np.zeros(max(1, n), dtype=_DESC_DTYPE)
    sizes = np.fromiter((g.U.size for g in gates), dtype=np.int64, count=n)
    if n:
        d["n_wires"][:n] = [len(g.wires) for g in gates]
        d["n_ctrl"][:n] = [len(g.controls) for g in gates]
        for i, g in enumerate(gates):
            k = len(g.wires)
            d["wires"][i, :k] = g.wires
            if g.controls:
                m = len(g.controls)
                d["ctrl_wires"][i, :m] = g.controls
                d["ctrl_vals"][i, :m] = g.values
        d["matrix_offset"][:n] = np.concatenate(([0], np.cumsum(sizes)[:-1]))
        m = np.concatenate([g.U.reshape(-1) for g in gates]).astype(np.complex128, copy=False)
    else:
        m = np.zeros(1, np.complex128)
    mats = np.ascontiguousarray(m).view(np.float64)
    descs = d.ctypes.data_as(ctypes.POINTER(qd_gate_desc))
    descs._keep = d  # the pointer keeps its buffer alive
    try:
        circuit._qd_arrays = (n, descs, mats)
    except AttributeError:
        pass
    return descs, mats


def _tc(tc_mode) -> int:
    return TC_MODES[tc_mode] if isinstance(tc_mode, str) else int(tc_mode)


def _opts(mode, max_tile_amps=0, min_gates=0, min_row=0, block_dim=0, tc_mode=QD_TC_TF32X3):
    if mode is None:
        return None
    return ctypes.byref(qd_fusion_opts(int(mode), int(max_tile_amps), int(min_gates), int(min_row), int(block_dim),
                                       _tc(tc_mode)))


def qd_apply_circuit(st: int, circuit, mode=QD_FUSE_OFF, max_tile_amps=0, min_gates=0, min_row=0,
                     block_dim=0, tc_mode=QD_TC_TF32X3) -> None:
    descs, m = circuit_arrays(circuit)
    _check(_lib.qd_apply_circuit(_vp(st), descs, len(circuit.gates), _p(m, _f64p),
                                 _opts(mode, max_tile_amps, min_gates, min_row, block_dim, tc_mode)),
           "qd_apply_circuit")


QD_SPARSE_MAX_NNZ = 512
QD_SPARSE_MAX_RESERVE = 1 << 22


def qd_sparse_create(dims, stream=None) -> int:
    d = _i32(dims)
    out = _vp()
    _check(_lib.qd_sparse_create(_p(d, _i32p), len(d), _vp(stream), ctypes.byref(out)), "qd_sparse_create")
    return out.value


def qd_sparse_destroy(s: int) -> None:
    _check(_lib.qd_sparse_destroy(_vp(s)), "qd_sparse_destroy")


def qd_sparse_run(s: int, circuit) -> None:
    descs, m = circuit_arrays(circuit)
    _check(_lib.qd_sparse_run(_vp(s), descs, len(circuit.gates), _p(m, _f64p)), "qd_sparse_run")


def qd_sparse_reserve(s: int, max_nnz: int) -> None:
    _check(_lib.qd_sparse_reserve(_vp(s), int(max_nnz)), "qd_sparse_reserve")


def qd_sparse_nnz(s: int) -> int:
    n = ctypes.c_int64()
    _check(_lib.qd_sparse_nnz(_vp(s), ctypes.byref(n)), "qd_sparse_nnz")
    return n.value


def qd_sparse_get(s: int) -> dict:
    """{basis index (Python int): complex amplitude}, ascending indices."""
    n = qd_sparse_nnz(s)
    lo = np.zeros(max(n, 1), dtype=np.uint64)
    hi = np.zeros(max(n, 1), dtype=np.uint64)
    amps = np.zeros(2 * max(n, 1), dtype=np.float64)
    got = ctypes.c_int64()
    _check(_lib.qd_sparse_get(_vp(s), lo.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                              hi.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _p(amps, _f64p), max(n, 1),
                              ctypes.byref(got)), "qd_sparse_get")
    return {int(lo[i]) + (int(hi[i]) << 64): complex(amps[2 * i], amps[2 * i + 1]) for i in range(got.value)}


def qd_set_fusion(st: int, max_block_dim: int, tc_mode=QD_TC_TF32X3) -> None:
    _check(_lib.qd_set_fusion(_vp(st), int(max_block_dim), _tc(tc_mode)), "qd_set_fusion")


def qd_set_lazy(st: int, enable: bool) -> None:
    _check(_lib.qd_set_lazy(_vp(st), 1 if enable else 0), "qd_set_lazy")


def qd_flush(st: int) -> None:
    _check(_lib.qd_flush(_vp(st)), "qd_flush")


def qd_plan_circuit(dims, prec, circuit, mode=QD_FUSE_TILE, max_tile_amps=0, min_gates=0, min_row=0, block_dim=0,
                    with_flops=False):
    """(exec_order, pass_of, pass_tile_amps[:n_passes]) of the circuit's execution plan,
    plus pass_flops[:n_passes] when ``with_flops``."""
    d = _i32(dims)
    descs, m = circuit_arrays(circuit)
    n = len(circuit.gates)
    order = np.zeros(max(1, n), np.int32)
    pass_of = np.zeros(max(1, n), np.int32)
    tiles = np.zeros(max(1, n), np.int64)
    flops = np.zeros(max(1, n), np.float64)
    npass = ctypes.c_int32()
    _check(_lib.qd_plan_circuit(_p(d, _i32p), len(d), prec, descs, n, _p(m, _f64p),
                                _opts(mode, max_tile_amps, min_gates, min_row, block_dim), _p(order, _i32p),
                                _p(pass_of, _i32p), tiles.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                _p(flops, _f64p), ctypes.byref(npass)), "qd_plan_circuit")
    if with_flops:
        return order[:n], pass_of[:n], tiles[:npass.value], flops[:npass.value]
    return order[:n], pass_of[:n], tiles[:npass.value]


def qd_batch_create(prec: int = QD_C64, stream: int = 0) -> int:
    out = _vp()
    _check(_lib.qd_batch_create(int(prec), _vp(stream), ctypes.byref(out)), "qd_batch_create")
    return out.value


QD_BATCH_LAYERS = 0   # eligible circuits through the device-side layer queue (default)
QD_BATCH_STREAMS = 1  # one program per circuit on auxiliary streams


def qd_batch_run(b: int, circuits, small_max_amps=0, n_streams=0, use_graph=False, fuse=True,
                 max_tile_amps=0, min_gates=0, min_row=0, block_dim=0, path=QD_BATCH_LAYERS) -> None:
    """Run independent circuits (each from |0...0>) as one batch; asynchronous."""
    n = len(circuits)
    arr = (qd_circuit * max(1, n))()
    keep = []
    for i, c in enumerate(circuits):
        dims = _i32(c.dims)
        descs, m = circuit_arrays(c)
        keep.append((dims, descs, m))
        arr[i].n_wires = len(dims)
        arr[i].dims = _p(dims, _i32p)
        arr[i].n_gates = len(c.gates)
        arr[i].gates = descs
        arr[i].matrices = _p(m, _f64p)
    opts = qd_batch_opts(int(small_max_amps), int(n_streams), 1 if use_graph else 0, int(path),
                         qd_fusion_opts(QD_FUSE_TILE if fuse else QD_FUSE_OFF, int(max_tile_amps), int(min_gates),
                                        int(min_row), int(block_dim), 0))
    _check(_lib.qd_batch_run(_vp(b), arr, n, ctypes.byref(opts)), "qd_batch_run")


def qd_batch_relaunch(b: int) -> None:
    _check(_lib.qd_batch_relaunch(_vp(b)), "qd_batch_relaunch")


def qd_batch_state(b: int, i: int):
    ptr = _vp()
    D = ctypes.c_int64()
    _check(_lib.qd_batch_state(_vp(b), int(i), ctypes.byref(ptr), ctypes.byref(D)), "qd_batch_state")
    return ptr.value, D.value


def qd_batch_get_amplitudes(b: int, i: int) -> np.ndarray:
    _, D = qd_batch_state(b, i)
    out = np.empty(D, dtype=np.complex128)
    _check(_lib.qd_batch_get_amplitudes(_vp(b), int(i), _p(out.view(np.float64), _f64p)), "qd_batch_get_amplitudes")
    return out


def qd_batch_norms(b: int, n: int) -> np.ndarray:
    out = np.empty(max(1, n), dtype=np.float64)
    _check(_lib.qd_batch_norms(_vp(b), _p(out, _f64p)), "qd_batch_norms")
    return out[:n]


def qd_batch_synchronize(b: int) -> None:
    _check(_lib.qd_batch_synchronize(_vp(b)), "qd_batch_synchronize")


def qd_batch_destroy(b: int) -> None:
    _check(_lib.qd_batch_destroy(_vp(b)), "qd_batch_destroy")


def _circuit_struct(c):
    dims = _i32(c.dims)
    descs, m = circuit_arrays(c)
    cs = qd_circuit(len(dims), _p(dims, _i32p), len(c.gates), descs, _p(m, _f64p))
    return cs, (dims, descs, m)


def qd_server_create(prec: int = QD_C64, hbm_budget_bytes: int = 0, max_slots: int = 0, small_max_amps: int = 0,
                     max_group: int = 0, fuse: bool = True, max_tile_amps: int = 0, block_dim: int = 0) -> int:
    opts = qd_server_opts(int(hbm_budget_bytes), int(max_slots), int(small_max_amps), int(max_group), 0,
                          qd_fusion_opts(QD_FUSE_TILE if fuse else QD_FUSE_OFF, int(max_tile_amps), 0, 0,
                                         int(block_dim), 0))
    out = _vp()
    _check(_lib.qd_server_create(int(prec), ctypes.byref(opts), ctypes.byref(out)), "qd_server_create")
    return out.value


def qd_server_submit(s: int, circuit, keep_state: bool = False) -> int:
    cs, keep = _circuit_struct(circuit)
    rid = ctypes.c_uint64()
    _check(_lib.qd_server_submit(_vp(s), ctypes.byref(cs), 1 if keep_state else 0, ctypes.byref(rid)),
           "qd_server_submit")
    return rid.value


def qd_server_submit_at(s: int, circuit, release_time: float, keep_state: bool = False) -> int:
    cs, keep = _circuit_struct(circuit)
    rid = ctypes.c_uint64()
    _check(_lib.qd_server_submit_at(_vp(s), ctypes.byref(cs), 1 if keep_state else 0, float(release_time),
                                    ctypes.byref(rid)), "qd_server_submit_at")
    return rid.value


def qd_server_poll(s: int, max_results: int = 4096):
    buf = (qd_request_result * max(1, max_results))()
    n = ctypes.c_int32()
    _check(_lib.qd_server_poll(_vp(s), buf, int(max_results), ctypes.byref(n)), "qd_server_poll")
    return [{f: getattr(buf[i], f) for f, _ in qd_request_result._fields_} for i in range(n.value)]


def qd_server_drain(s: int, timeout_s: float = 600.0) -> None:
    _check(_lib.qd_server_drain(_vp(s), float(timeout_s)), "qd_server_drain")


def qd_server_now(s: int) -> float:
    t = ctypes.c_double()
    _check(_lib.qd_server_now(_vp(s), ctypes.byref(t)), "qd_server_now")
    return t.value


def qd_server_get_amplitudes(s: int, rid: int, num_amplitudes: int) -> np.ndarray:
    out = np.empty(int(num_amplitudes), dtype=np.complex128)
    _check(_lib.qd_server_get_amplitudes(_vp(s), int(rid), _p(out.view(np.float64), _f64p)),
           "qd_server_get_amplitudes")
    return out


def qd_server_release(s: int, rid: int) -> None:
    _check(_lib.qd_server_release(_vp(s), int(rid)), "qd_server_release")


def qd_server_destroy(s: int) -> None:
    _check(_lib.qd_server_destroy(_vp(s)), "qd_server_destroy")


# --- convenience ----------------------------------------------------------------------------------
class State:
    """A state vector in torch-allocated device memory, driven through the C ABI.

    ``prec`` is ``QD_C64`` or ``QD_C128``.  Work is issued on ``stream``
    (a ``torch.cuda.Stream``; default: the current stream at creation).
    """

    def __init__(self, dims: Sequence[int], prec: int = QD_C128, stream=None, device: int = 0):
        import torch

        self.dims = tuple(int(x) for x in dims)
        self.prec = prec
        self.D = int(np.prod(np.asarray(self.dims, dtype=np.int64)))
        dt = torch.float32 if prec == QD_C64 else torch.float64
        torch.cuda.set_device(device)
        self.buf = torch.empty(2 * self.D, dtype=dt, device=f"cuda:{device}")
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.handle = qd_state_wrap(self.buf.data_ptr(), self.buf.numel() * self.buf.element_size(), self.dims,
                                    prec, self.stream.cuda_stream)
        qd_state_reset(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            qd_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        qd_state_reset(self.handle)

    def apply(self, gate) -> None:
        """Apply an ``inputs.Gate``."""
        if len(gate.wires) == 1 and not gate.controls:
            qd_apply_gate(self.handle, gate.wires[0], gate.U)
        elif len(gate.wires) == 1:
            qd_apply_controlled(self.handle, gate.wires[0], gate.U, gate.controls, gate.values)
        else:
            qd_apply_multi(self.handle, gate.wires, gate.U, gate.controls, gate.values)

    def run(self, circuit, fuse=False, **opts) -> None:
        """Apply the circuit's gates through one qd_apply_circuit call.  ``fuse``:
        False / "off" (one pass per gate), True / "tile" (shared-memory tile
        passes) or "block" (composed blocks over the whole state, tensor cores
        for large complex64 blocks; ``tc_mode`` "tf32x3" / "bf16x3" / "fp32")."""
        mode = {False: QD_FUSE_OFF, "off": QD_FUSE_OFF, True: QD_FUSE_TILE, "tile": QD_FUSE_TILE,
                "block": QD_FUSE_BLOCK}[fuse]
        qd_apply_circuit(self.handle, circuit, mode, **opts)

    def set_fusion(self, max_block_dim: int, tc_mode=QD_TC_TF32X3) -> None:
        """Deferred fusion of ``apply`` calls (``max_block_dim`` <= 1: off);
        ``tc_mode``: "tf32x3", "bf16x3", "fp32" or a QD_TC_* value."""
        qd_set_fusion(self.handle, max_block_dim, tc_mode)

    def flush(self) -> None:
        qd_flush(self.handle)

    def set_lazy(self, enable: bool = True) -> None:
        """Fold single-wire phase / permutation gates into a per-wire frame (no launch)."""
        qd_set_lazy(self.handle, enable)

    def run_gate_by_gate(self, circuit) -> None:
        for g in circuit.gates:
            self.apply(g)

    def amplitudes(self) -> np.ndarray:
        return qd_state_get_amplitudes(self.handle)

    def raw(self) -> np.ndarray:
        return qd_state_get_raw(self.handle)

    def set_amplitudes(self, psi) -> None:
        qd_state_set_amplitudes(self.handle, psi)

    def norm(self) -> float:
        return qd_norm(self.handle)

    def probabilities(self) -> np.ndarray:
        return qd_probabilities(self.handle)

    def marginal(self, wire: int) -> np.ndarray:
        return qd_marginal(self.handle, wire, self.dims[wire])

    def synchronize(self) -> None:
        qd_synchronize(self.handle)
