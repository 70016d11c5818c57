"""Python driver for the reference oracle (``oracle.c``).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT: only the tests, the smoke check
and the CPU-baseline leg of the benchmark may import this module. It shares no
code with the CUDA path; the only thing both sides use is the seeded input
generator module, which holds no arithmetic of the method.

The circuit definitions here are the oracle's own:

* Hardware-efficient ansatz (HEA): each of the ``d`` layers applies RZ, RY, RZ
  on every qubit and then a chain of CZ gates (0,1), (1,2), ..., (n-2, n-1)
  (a ring adds (n-1, 0)). Parameter index of gate g in {0: first RZ, 1: RY,
  2: second RZ} on qubit q in layer l is ``l*3n + 3q + g``.
* Data encoding: RY(x_q) on qubit q of |0...0>, before layer 0; x is not
  trainable.
* Loss reading: ``L = sum_b E_b`` (the paper's L = E, Sec. 2.1) or the mean
  squared error ``L = mean_b (E_b - y_b)^2``; dL/dE_b enters the adjoint seed
  through the chain rule (Eq. 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RX, RY, RZ, CZ, CNOT = 0, 1, 2, 3, 4
PAULI = {"I": 0, "X": 1, "Y": 2, "Z": 3}


class _Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32),
                ("q1", ctypes.c_int32), ("param", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        gp = ctypes.POINTER(_Gate)
        lib.oracle_final_state.argtypes = [ctypes.c_int, gp, ctypes.c_int, dp, dp, dp, dp]
        lib.oracle_expectation.argtypes = [ctypes.c_int, gp, ctypes.c_int, dp, ctypes.c_int,
                                           dp, dp, ip, dp, ctypes.c_int]
        lib.oracle_gradient.argtypes = [ctypes.c_int, gp, ctypes.c_int, dp, ctypes.c_int,
                                        ctypes.c_int, dp, dp, ip, dp, ctypes.c_int,
                                        ctypes.c_int, dp, dp, ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Circuit:
    """A gate list for the oracle: rows of (kind, q0, q1, param)."""
    n: int
    gates: np.ndarray  # int32 [M, 4]
    n_params: int


def hea(n: int, d: int, entangler: str = "chain",
        rotations: tuple[int, int, int] = (RZ, RY, RZ)) -> Circuit:
    """The hardware-efficient ansatz, gate by gate, in circuit order."""
    rows = []
    for l in range(d):
        for q in range(n):
            for g, kind in enumerate(rotations):
                rows.append((kind, q, -1, l * 3 * n + 3 * q + g))
        for q in range(n - 1):
            rows.append((CZ, q, q + 1, -1))
        if entangler == "ring" and n > 2:
            rows.append((CZ, n - 1, 0, -1))
    gates = np.array(rows, dtype=np.int32).reshape(-1, 4)
    return Circuit(n=n, gates=gates, n_params=3 * n * d)


def pauli_letters(n: int, obs: str | dict) -> np.ndarray:
    """Observable as one Pauli letter per qubit.

    ``obs`` is either a string over {I,X,Y,Z} whose k-th character acts on
    qubit k, or a dict {qubit: letter}.
    """
    letters = np.zeros(n, dtype=np.int32)
    if isinstance(obs, dict):
        for q, ch in obs.items():
            letters[q] = PAULI[ch]
    else:
        for q, ch in enumerate(obs):
            letters[q] = PAULI[ch]
    return letters


def _gates_ptr(c: Circuit):
    g = np.ascontiguousarray(c.gates, dtype=np.int32)
    arr = (_Gate * max(len(g), 1))()
    for i, (k, a, b, p) in enumerate(g):
        arr[i] = _Gate(int(k), int(a), int(b), int(p))
    return arr


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def final_state(c: Circuit, theta, x=None, init_state=None) -> np.ndarray:
    """psi_M of one sample as complex128 [2^n]."""
    lib = _load()
    theta = _f64(theta)
    x = _f64(x)
    init = None if init_state is None else _f64(np.stack([np.real(init_state), np.imag(init_state)], -1))
    out = np.zeros(2 << c.n, dtype=np.float64)
    rc = lib.oracle_final_state(c.n, _gates_ptr(c), len(c.gates), _dptr(theta), _dptr(x),
                                _dptr(init), _dptr(out))
    if rc != 0:
        raise MemoryError("oracle_final_state failed")
    return out[0::2] + 1j * out[1::2]


def expectation(c: Circuit, theta, x, obs="Z", init_states=None, threads: int = 0) -> np.ndarray:
    """E_b (Eq. 1) for every sample: x is [B][n] (or init_states [B][2^n])."""
    lib = _load()
    theta = _f64(theta)
    B = len(x) if x is not None else len(init_states)
    x = _f64(x)
    init = None if init_states is None else _f64(
        np.stack([np.real(init_states), np.imag(init_states)], -1))
    letters = pauli_letters(c.n, obs)
    E = np.zeros(B, dtype=np.float64)
    rc = lib.oracle_expectation(c.n, _gates_ptr(c), len(c.gates), _dptr(theta), B, _dptr(x),
                                _dptr(init), letters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                _dptr(E), int(threads))
    if rc != 0:
        raise MemoryError("oracle_expectation failed")
    return E


def gradient(c: Circuit, theta, x, obs="Z", dLdE=None, per_sample: bool = False,
             block: int = 0, init_states=None, threads: int = 0):
    """Adjoint gradients (Eqs. 2-4). Returns (grad, E).

    grad is [n_params] (summed over samples) or [B][n_params] when per_sample.
    dLdE defaults to ones (L = sum_b E_b). block = gates per recompute block
    (0 picks about sqrt(M)).
    """
    lib = _load()
    theta = _f64(theta)
    B = len(x) if x is not None else len(init_states)
    x = _f64(x)
    init = None if init_states is None else _f64(
        np.stack([np.real(init_states), np.imag(init_states)], -1))
    letters = pauli_letters(c.n, obs)
    dLdE = np.ones(B) if dLdE is None else _f64(dLdE)
    M = len(c.gates)
    if block <= 0:
        block = max(1, int(np.ceil(np.sqrt(max(M, 1)))))
    grad = np.zeros((B, c.n_params) if per_sample else c.n_params, dtype=np.float64)
    E = np.zeros(B, dtype=np.float64)
    rc = lib.oracle_gradient(c.n, _gates_ptr(c), M, _dptr(theta), c.n_params, B, _dptr(x),
                             _dptr(init), letters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             _dptr(dLdE), int(per_sample), int(block), _dptr(grad), _dptr(E),
                             int(threads))
    if rc != 0:
        raise MemoryError("oracle_gradient failed")
    return grad, E


def mse_loss(E, y) -> float:
    """L = mean_b (E_b - y_b)^2."""
    E = np.asarray(E, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean((E - y) ** 2))


def mse_dLdE(E, y) -> np.ndarray:
    """dL/dE_b = 2 (E_b - y_b) / B for the mean squared error."""
    E = np.asarray(E, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return 2.0 * (E - y) / len(E)


def max_threads() -> int:
    return int(_load().oracle_max_threads())
