"""Seeded synthetic workloads.

This module only draws random inputs. It holds none of the simulation's
arithmetic, so both the CUDA path and the reference oracle can take their
inputs from it.

RNG: numpy ``default_rng`` (PCG64) with fixed seeds. Values are drawn in
float64 and cast to float32; the same float32 arrays feed both sides (the
oracle promotes them exactly to float64).

Named workloads (hardware-efficient ansatz: RZ, RY, RZ on every qubit, then a
CZ chain; RY(x) data encoding; observable Z on qubit 0):

======== ===== ====== ====== ======================================== =========
name      n     d      B      values                                   seeds
======== ===== ====== ====== ======================================== =========
tiny      4     2      8      theta~U[0,2pi), x~U[0,pi]^4, L=sum E     101, 201
hea12     12    20     256    as tiny, y~{-1,+1}, L=MSE                102,202,302
hea16     16    100    128    as hea12, checkpoint every 10 layers     103,203,303
mixed512  8-18  10-200 1-64   512 circuits, L=sum E                    104 (+id)
hea20     20    1000   1000   micro-batched, L=sum E                   105, 205
======== ===== ====== ====== ======================================== =========
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * np.pi


@dataclass
class Workload:
    name: str
    n: int
    d: int
    B: int
    loss: str = "sum"          # "sum": L = sum_b E_b ; "mse": L = mean_b (E_b - y_b)^2
    obs: str = "Z"             # Pauli string, character k acts on qubit k
    seeds: tuple = (0, 0, 0)   # (theta, x, y)
    ckpt_layers: int = 0       # checkpoint interval in layers (0 = chosen by the library)
    extra: dict = field(default_factory=dict)

    @property
    def n_params(self) -> int:
        return 3 * self.n * self.d


WORKLOADS = {
    "tiny": Workload("tiny", 4, 2, 8, "sum", "Z", (101, 201, 0)),
    "hea12": Workload("hea12", 12, 20, 256, "mse", "Z", (102, 202, 302)),
    "hea16": Workload("hea16", 16, 100, 128, "mse", "Z", (103, 203, 303), ckpt_layers=10,
                      extra={"fd_seed": 402, "fd_params": 32, "fd_h": 1e-3}),
    "hea20": Workload("hea20", 20, 1000, 1000, "sum", "Z", (105, 205, 0)),
}


def draw_theta(n_params: int, seed: int) -> np.ndarray:
    """theta ~ U[0, 2pi), float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, TWO_PI, size=n_params).astype(np.float32)


def draw_x(B: int, n: int, seed: int) -> np.ndarray:
    """Encoding angles x ~ U[0, pi]^n per sample, float32 [B, n]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, np.pi, size=(B, n)).astype(np.float32)


def draw_labels(B: int, seed: int) -> np.ndarray:
    """Labels y ~ uniform over {-1, +1}, float32 [B]."""
    rng = np.random.default_rng(seed)
    return (2 * rng.integers(0, 2, size=B) - 1).astype(np.float32)


def draw_state(B: int, n: int, seed: int, dtype=np.complex64) -> np.ndarray:
    """Random normalised initial states (complex Gaussian), [B, 2^n] of
    `dtype` (complex64, or complex128 for complex128 plans)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((B, 1 << n)) + 1j * rng.standard_normal((B, 1 << n))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return z.astype(dtype)


def make_inputs(w: Workload, B: int | None = None):
    """(theta [P] f32, x [B, n] f32, y [B] f32 or None) for a named workload.

    B overrides the batch size; the first B rows of the full draw are used so
    a smaller batch is a prefix of the full one.
    """
    theta = draw_theta(w.n_params, w.seeds[0])
    x = draw_x(w.B, w.n, w.seeds[1])
    y = draw_labels(w.B, w.seeds[2]) if w.loss == "mse" else None
    if B is not None:
        if B <= w.B:
            x = x[:B]
            y = None if y is None else y[:B]
        else:
            x = draw_x(B, w.n, w.seeds[1])
            y = None if y is None else draw_labels(B, w.seeds[2])
    return theta, x, y


def draw_fd_params(n_params: int, count: int, seed: int) -> np.ndarray:
    """Indices of the parameters checked by finite differences."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_params, size=count, replace=False)).astype(np.int64)


@dataclass
class MixedCircuit:
    cid: int
    n: int
    d: int
    B: int
    theta: np.ndarray
    x: np.ndarray


def mixed_circuits(count: int = 512, seed: int = 104, n_range=(8, 18), d_range=(10, 200),
                   b_range=(1, 64), with_values: bool = True) -> list[MixedCircuit]:
    """Uneven batch of HEA circuits: n ~ U{8..18}, d ~ U{10..200}, B ~ U{1..64}.

    The structure is drawn with ``seed``; circuit ``i`` draws theta and x with
    seed ``seed + i`` (theta first, then x, from one generator).
    """
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    ds = rng.integers(d_range[0], d_range[1] + 1, size=count)
    bs = rng.integers(b_range[0], b_range[1] + 1, size=count)
    out = []
    for i in range(count):
        n, d, B = int(ns[i]), int(ds[i]), int(bs[i])
        if with_values:
            r = np.random.default_rng(seed + i)
            theta = r.uniform(0.0, TWO_PI, size=3 * n * d).astype(np.float32)
            x = r.uniform(0.0, np.pi, size=(B, n)).astype(np.float32)
        else:
            theta = np.zeros(0, np.float32)
            x = np.zeros((0, n), np.float32)
        out.append(MixedCircuit(i, n, d, B, theta, x))
    return out


def xyz_ring_gates(n: int, d: int) -> list[tuple[int, int, int, int]]:
    """The ansatz of the paper's throughput measurements (Sec. 4.2): every
    layer applies Rx, Ry, Rz to every qubit, then CZ(q, q+1) for q < n-1 and
    CZ(n-1, 0) (a ring; for n = 2 the single CZ). Rows (kind, q0, q1, param)
    with kinds 0 RX, 1 RY, 2 RZ, 3 CZ; parameter l*3n + 3q + g, g in
    {0: Rx, 1: Ry, 2: Rz}."""
    rows = []
    for layer in range(d):
        for q in range(n):
            for g in range(3):
                rows.append((g, q, -1, layer * 3 * n + 3 * q + g))
        for q in range(n - 1):
            rows.append((3, q, q + 1, -1))
        if n > 2:
            rows.append((3, n - 1, 0, -1))
    return rows


def ixyz(n: int) -> str:
    """O = IXYZ IXYZ ... truncated to n letters, letter k on qubit k (Sec. 4.2)."""
    return ("IXYZ" * ((n + 3) // 4))[:n]


def consecutive_gates(n: int, m: int) -> list[tuple[int, int, int, int]]:
    """The fusion-depth circuit of Sec. 4.1: m consecutive single-qubit gates on
    every qubit in the repeating order Rx, Ry, Rz (no entangler); parameter
    q*m + k for the k-th gate on qubit q. Rows as in xyz_ring_gates."""
    return [(k % 3, q, -1, q * m + k) for q in range(n) for k in range(m)]
