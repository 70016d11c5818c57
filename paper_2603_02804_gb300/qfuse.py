"""ctypes binding of the C-ABI in ``include/qfuse.h``.

Argument marshalling only: every function here has the name of the C entry
point it calls and forwards plain pointers and sizes. Tensors may be passed
wherever a device pointer is expected (their ``data_ptr()`` is used). The
library must have been built (``paper_2603_02804_gb300.build.build()``);
loading fails loudly otherwise, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqfuse.so")

QF_OK, QF_ERR_INVALID_ARG, QF_ERR_UNSUPPORTED, QF_ERR_WORKSPACE, QF_ERR_OOM, QF_ERR_CUDA, QF_ERR_TIMEOUT = range(7)
QF_GATE_RX, QF_GATE_RY, QF_GATE_RZ, QF_GATE_CZ, QF_GATE_CNOT = range(5)
QF_ENT_CHAIN, QF_ENT_RING = 0, 1
QF_ENC_RY_X, QF_ENC_STATE_IN = 0, 1
QF_PATH_FUSED, QF_PATH_PER_GATE = 0, 1
QF_LOSS_SUM, QF_LOSS_MSE = 0, 1
QF_PREC_C64, QF_PREC_C128 = 0, 1

STATUS_NAMES = {0: "QF_OK", 1: "QF_ERR_INVALID_ARG", 2: "QF_ERR_UNSUPPORTED", 3: "QF_ERR_WORKSPACE",
                4: "QF_ERR_OOM", 5: "QF_ERR_CUDA", 6: "QF_ERR_TIMEOUT"}


class QFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class qf_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("param", ctypes.c_int32)]


class qf_pauli(ctypes.Structure):
    _fields_ = [("x_mask", ctypes.c_uint64), ("z_mask", ctypes.c_uint64)]


class qf_plan_opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("tile_bits", ctypes.c_int32), ("ckpt_layers", ctypes.c_int32),
                ("host_only", ctypes.c_int32), ("program", ctypes.c_int32), ("ckpt_mode", ctypes.c_int32),
                ("mem_save", ctypes.c_int32), ("tc_path", ctypes.c_int32), ("no_host_staging", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("catch_up", ctypes.c_int32), ("fwd_ctas", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class qf_plan_info_t(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "n_qubits", "n_eff", "n_params", "n_slots", "path", "tile_bits", "n_passes", "n_steps",
        "n_fused_ops", "n_ckpt", "ckpt_layers", "launches_fwd", "launches_bwd")] + [
        ("batch", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64), ("state_bytes", ctypes.c_int64)] + [
        (name, ctypes.c_int32) for name in ("ckpt_mode", "mem_save", "n_pass_slots", "tc_path", "precision",
                                            "qubit_shift", "catch_up", "fwd_ctas")]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t

# C signature table: name -> (argtypes, restype)
SIGNATURES = {
    "qf_hea_create": ([_i32, _i32, _i32, _i32, ctypes.POINTER(_vp)], _i32),
    "qf_circuit_create": ([_i32, ctypes.POINTER(qf_gate), _i32, _i32, _i32, ctypes.POINTER(_vp)], _i32),
    "qf_circuit_destroy": ([_vp], _i32),
    "qf_plan": ([_vp, ctypes.POINTER(qf_plan_opts), _i64, ctypes.POINTER(_sz)], _i32),
    "qf_plan_info": ([_vp, ctypes.POINTER(qf_plan_info_t)], _i32),
    "qf_mem_model": ([ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
                     ctypes.c_double),
    "qf_plan_fit": ([_vp, ctypes.POINTER(qf_plan_opts), _i64, _sz, ctypes.POINTER(_i32), ctypes.POINTER(_sz)],
                    _i32),
    "qf_plan_export": ([_vp, _i32, ctypes.POINTER(_i32), _i64, ctypes.POINTER(_i64)], _i32),
    "qf_forward": ([_vp, _vp, _vp, _i64, qf_pauli, _vp, _vp, _sz, _vp], _i32),
    "qf_backward": ([_vp, _vp, _vp, _i64, qf_pauli, _vp, _vp, _i32, _vp, _sz, _vp], _i32),
    "qf_loss": ([_i32, _vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "qf_train_step": ([_vp, _vp, _vp, _vp, _i64, _i32, qf_pauli, _vp, _vp, _vp, _vp, _sz, _vp], _i32),
    "qf_train_step_host": ([_vp, _vp, _vp, _vp, _i64, _i32, qf_pauli, _vp, _vp, _vp, _vp, _sz, _vp], _i32),
    "qf_train_step_noalloc": ([_vp, _vp, _vp, _vp, _i64, _i32, qf_pauli, _vp, _vp, _vp, _vp], _i32),
    "qf_forward64": ([_vp, _vp, _vp, _i64, qf_pauli, _vp, _vp, _sz, _vp], _i32),
    "qf_backward64": ([_vp, _vp, _vp, _i64, qf_pauli, _vp, _vp, _i32, _vp, _sz, _vp], _i32),
    "qf_loss64": ([_i32, _vp, _vp, _i64, _vp, _vp, _vp], _i32),
    "qf_train_step64": ([_vp, _vp, _vp, _vp, _i64, _i32, qf_pauli, _vp, _vp, _vp, _vp, _sz, _vp], _i32),
    "qf_train_step_host64": ([_vp, _vp, _vp, _vp, _i64, _i32, qf_pauli, _vp, _vp, _vp, _vp, _sz, _vp], _i32),
    "qf_batch_create": ([_i32, ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(qf_pauli), _i32,
                         ctypes.POINTER(_sz), ctypes.POINTER(_vp)], _i32),
    "qf_batch_layout": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _i32),
    "qf_batch_train_step": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i32),
    "qf_batch_graph_capture": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i32),
    "qf_batch_graph_launch": ([_vp, _vp], _i32),
    "qf_batch_info": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _i32),
    "qf_batch_destroy": ([_vp], _i32),
    "qf_launch_count": ([_vp, ctypes.POINTER(_i64)], _i32),
    "qf_graph_stats": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _i32),
    "qf_profile": ([_vp, _i32], _i32),
    "qf_profile_read": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)], _i32),
    "qf_device_status": ([_vp, ctypes.POINTER(_i32)], _i32),
    "qf_check_bounded_wait": ([_vp, _i64], _i32),
    "qf_last_error": ([], ctypes.c_char_p),
    "qf_version": ([], _i32),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libqfuse.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2603_02804_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _ptr(t) -> int | None:
    """Device/host address of a tensor, numpy array or int (None stays NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def _check(status: int):
    if status != QF_OK:
        raise QFError(status, load().qf_last_error().decode())


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def pauli(obs, n: int) -> qf_pauli:
    """Observable from a string over {I,X,Y,Z} (character k acts on qubit k)
    or a dict {qubit: letter}."""
    items = obs.items() if isinstance(obs, dict) else enumerate(obs)
    x = z = 0
    for q, ch in items:
        if q >= n:
            raise ValueError("observable longer than the circuit")
        if ch in "XY":
            x |= 1 << q
        if ch in "ZY":
            z |= 1 << q
        if ch not in "IXYZ":
            raise ValueError(f"bad Pauli letter {ch!r}")
    return qf_pauli(x, z)


# ---- entry points (same names as the C-ABI) -------------------------------------
def qf_hea_create(n_qubits: int, n_layers: int, entangler: int = QF_ENT_CHAIN, encoding: int = QF_ENC_RY_X) -> int:
    h = _vp()
    _check(load().qf_hea_create(n_qubits, n_layers, entangler, encoding, ctypes.byref(h)))
    return h.value


def qf_circuit_create(n_qubits: int, gates, n_params: int, encoding: int = QF_ENC_RY_X) -> int:
    arr = (qf_gate * max(len(gates), 1))(*[qf_gate(*map(int, g)) for g in gates])
    h = _vp()
    _check(load().qf_circuit_create(n_qubits, arr, len(gates), n_params, encoding, ctypes.byref(h)))
    return h.value


def qf_circuit_destroy(handle: int) -> None:
    _check(load().qf_circuit_destroy(handle))


def qf_plan(handle: int, batch: int, path: int = QF_PATH_FUSED, tile_bits: int = 0, ckpt_layers: int = 0,
            host_only: bool = False, program: int = 0, ckpt_mode: int = 0, mem_save: bool = False,
            tc_path: bool = False, host_staging: bool = True, precision: int = QF_PREC_C64, catch_up: int = 0,
            fwd_ctas: int = 0) -> int:
    o = qf_plan_opts(path, tile_bits, ckpt_layers, int(host_only), int(program), int(ckpt_mode), int(mem_save),
                     int(tc_path), int(not host_staging), int(precision), int(catch_up), int(fwd_ctas))
    ws = _sz()
    _check(load().qf_plan(handle, ctypes.byref(o), batch, ctypes.byref(ws)))
    return ws.value


def qf_mem_model(k: float, d: float, b: float):
    """(stored state vectors k b + d / b, minimising block size sqrt(d / k))."""
    best = ctypes.c_double()
    m = load().qf_mem_model(float(k), float(d), float(b), ctypes.byref(best))
    return m, best.value


def qf_plan_fit(handle: int, batch: int, mem_bytes: int, path: int = QF_PATH_FUSED, tile_bits: int = 0,
                host_only: bool = False, program: int = 0, ckpt_mode: int = 0, mem_save: bool = False,
                tc_path: bool = False, host_staging: bool = True, precision: int = QF_PREC_C64, catch_up: int = 0,
                fwd_ctas: int = 0):
    """Plan with a checkpoint interval that fits mem_bytes (mode 0: the smallest;
    mode 1: the one with the smallest workspace): (c, workspace bytes)."""
    o = qf_plan_opts(path, tile_bits, 0, int(host_only), int(program), int(ckpt_mode), int(mem_save),
                     int(tc_path), int(not host_staging), int(precision), int(catch_up), int(fwd_ctas))
    c = _i32()
    ws = _sz()
    _check(load().qf_plan_fit(handle, ctypes.byref(o), batch, mem_bytes, ctypes.byref(c), ctypes.byref(ws)))
    return c.value, ws.value


def qf_plan_info(handle: int) -> dict:
    info = qf_plan_info_t()
    _check(load().qf_plan_info(handle, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in qf_plan_info_t._fields_}


def qf_plan_export(handle: int, direction: int):
    import numpy as np
    n = _i64()
    _check(load().qf_plan_export(handle, direction, None, 0, ctypes.byref(n)))
    buf = np.zeros(n.value, dtype=np.int32)
    _check(load().qf_plan_export(handle, direction, buf.ctypes.data_as(ctypes.POINTER(_i32)), n.value,
                                 ctypes.byref(n)))
    return buf


def qf_forward(handle, theta, x, batch, obs: qf_pauli, E, ws, ws_bytes, stream=None) -> None:
    _check(load().qf_forward(handle, _ptr(theta), _ptr(x), batch, obs, _ptr(E), _ptr(ws), ws_bytes,
                             _stream(stream)))


def qf_backward(handle, theta, x, batch, obs: qf_pauli, dLdE, grad, per_sample, ws, ws_bytes, stream=None) -> None:
    _check(load().qf_backward(handle, _ptr(theta), _ptr(x), batch, obs, _ptr(dLdE), _ptr(grad), int(per_sample),
                              _ptr(ws), ws_bytes, _stream(stream)))


def qf_loss(kind, E, y, batch, loss, dLdE, stream=None) -> None:
    _check(load().qf_loss(kind, _ptr(E), _ptr(y), batch, _ptr(loss), _ptr(dLdE), _stream(stream)))


def qf_train_step(handle, theta, x, y, batch, loss_kind, obs, loss, E, grad, ws, ws_bytes, stream=None) -> None:
    _check(load().qf_train_step(handle, _ptr(theta), _ptr(x), _ptr(y), batch, loss_kind, obs, _ptr(loss), _ptr(E),
                                _ptr(grad), _ptr(ws), ws_bytes, _stream(stream)))


def qf_train_step_host(handle, theta, x, y, batch, loss_kind, obs, loss, E, grad, ws, ws_bytes, stream=None):
    _check(load().qf_train_step_host(handle, _ptr(theta), _ptr(x), _ptr(y), batch, loss_kind, obs, _ptr(loss),
                                     _ptr(E), _ptr(grad), _ptr(ws), ws_bytes, _stream(stream)))


def qf_train_step_noalloc(handle, theta, x, y, batch, loss_kind, obs, loss, E, grad, stream=None) -> None:
    _check(load().qf_train_step_noalloc(handle, _ptr(theta), _ptr(x), _ptr(y), batch, loss_kind, obs, _ptr(loss),
                                        _ptr(E), _ptr(grad), _stream(stream)))


QF_NOALLOC_MAX_BYTES = 32 * 1024 * 1024


# complex128 plans (precision=QF_PREC_C128): float64 theta, x, y
def qf_forward64(handle, theta, x, batch, obs: qf_pauli, E, ws, ws_bytes, stream=None) -> None:
    _check(load().qf_forward64(handle, _ptr(theta), _ptr(x), batch, obs, _ptr(E), _ptr(ws), ws_bytes,
                               _stream(stream)))


def qf_backward64(handle, theta, x, batch, obs: qf_pauli, dLdE, grad, per_sample, ws, ws_bytes,
                  stream=None) -> None:
    _check(load().qf_backward64(handle, _ptr(theta), _ptr(x), batch, obs, _ptr(dLdE), _ptr(grad), int(per_sample),
                                _ptr(ws), ws_bytes, _stream(stream)))


def qf_loss64(kind, E, y, batch, loss, dLdE, stream=None) -> None:
    _check(load().qf_loss64(kind, _ptr(E), _ptr(y), batch, _ptr(loss), _ptr(dLdE), _stream(stream)))


def qf_train_step64(handle, theta, x, y, batch, loss_kind, obs, loss, E, grad, ws, ws_bytes, stream=None) -> None:
    _check(load().qf_train_step64(handle, _ptr(theta), _ptr(x), _ptr(y), batch, loss_kind, obs, _ptr(loss),
                                  _ptr(E), _ptr(grad), _ptr(ws), ws_bytes, _stream(stream)))


def qf_train_step_host64(handle, theta, x, y, batch, loss_kind, obs, loss, E, grad, ws, ws_bytes, stream=None):
    _check(load().qf_train_step_host64(handle, _ptr(theta), _ptr(x), _ptr(y), batch, loss_kind, obs, _ptr(loss),
                                       _ptr(E), _ptr(grad), _ptr(ws), ws_bytes, _stream(stream)))


def qf_batch_create(circuits, batch, obs, loss_kind=QF_LOSS_SUM):
    """Returns (batch handle, workspace bytes)."""
    n = len(circuits)
    hs = (_vp * n)(*circuits)
    bs = (_i64 * n)(*[int(v) for v in batch])
    ob = (qf_pauli * n)(*obs)
    ws = _sz()
    h = _vp()
    _check(load().qf_batch_create(n, hs, bs, ob, loss_kind, ctypes.byref(ws), ctypes.byref(h)))
    return h.value, ws.value


def qf_batch_layout(handle, n):
    t, x, s = (_i64 * (n + 1))(), (_i64 * (n + 1))(), (_i64 * (n + 1))()
    _check(load().qf_batch_layout(handle, t, x, s))
    return list(t), list(x), list(s)


def qf_batch_train_step(handle, theta, x, y, loss, E, grad, ws, ws_bytes, stream=None) -> None:
    _check(load().qf_batch_train_step(handle, _ptr(theta), _ptr(x), _ptr(y), _ptr(loss), _ptr(E), _ptr(grad),
                                      _ptr(ws), ws_bytes, _stream(stream)))


def qf_batch_graph_capture(handle, theta, x, y, loss, E, grad, ws, ws_bytes, stream) -> None:
    _check(load().qf_batch_graph_capture(handle, _ptr(theta), _ptr(x), _ptr(y), _ptr(loss), _ptr(E), _ptr(grad),
                                         _ptr(ws), ws_bytes, _stream(stream)))


def qf_batch_graph_launch(handle, stream) -> None:
    _check(load().qf_batch_graph_launch(handle, _stream(stream)))


def qf_batch_info(handle) -> dict:
    a, b, c = _i64(), _i64(), _i64()
    _check(load().qf_batch_info(handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"n_items": a.value, "n_samples": b.value, "n_params": c.value}


def qf_batch_destroy(handle) -> None:
    _check(load().qf_batch_destroy(handle))


def qf_launch_count(handle) -> int:
    n = _i64()
    _check(load().qf_launch_count(handle, ctypes.byref(n)))
    return n.value


def qf_graph_stats(handle) -> dict:
    """Train steps recorded as CUDA graphs and replayed from one by this handle."""
    rec, rep = _i64(), _i64()
    _check(load().qf_graph_stats(handle, ctypes.byref(rec), ctypes.byref(rep)))
    return {"recorded": rec.value, "replayed": rep.value}


def qf_profile(handle, on: bool) -> None:
    _check(load().qf_profile(handle, int(on)))


def qf_profile_read(handle) -> dict:
    fm, bm = ctypes.c_double(), ctypes.c_double()
    fl, bl = _i64(), _i64()
    _check(load().qf_profile_read(handle, ctypes.byref(fm), ctypes.byref(fl), ctypes.byref(bm), ctypes.byref(bl)))
    return {"fwd_ms": fm.value, "fwd_launches": fl.value, "bwd_ms": bm.value, "bwd_launches": bl.value}


def qf_device_status(stream=None) -> int:
    """Read and clear the device error word (0: none; 1: a bounded wait gave up)."""
    code = _i32()
    _check(load().qf_device_status(_stream(stream), ctypes.byref(code)))
    return code.value


def qf_check_bounded_wait(spin_limit: int, stream=None) -> None:
    """Launch one bounded wait that times out (records 1 in the device error word)."""
    _check(load().qf_check_bounded_wait(_stream(stream), spin_limit))


def qf_last_error() -> str:
    return load().qf_last_error().decode()


def qf_version() -> int:
    return load().qf_version()
