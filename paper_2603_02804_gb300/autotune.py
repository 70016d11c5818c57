"""Autotuner for the fused path's tile width.

For circuits wider than one tile (n > 12), the tile width K (qubits held in
shared memory per pass) trades HBM passes against full register rounds; only
widths whose non-low part is a whole number of 4-qubit chunks give padding-free
round programs, so the candidates are K in {8, 12} (plus any the caller adds).
For each (GPU, n, depth bucket, batch bucket) the tuner times
qf_train_step for every candidate on synthetic inputs and keeps the fastest
in a JSON cache. Circuits with n <= 12 hold the whole state (K = n).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import workloads
from .torch_api import Simulator

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "qfuse", "autotune.json")
CANDIDATES = (12, 8)


def bucket(v: int) -> int:
    """Power-of-two bucket (1, 2, 4, ...)."""
    return 1 << max(0, math.ceil(math.log2(max(1, v))))


def key(n: int, d: int, B: int) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|n={n}|d~{bucket(d)}|B~{bucket(B)}"


class Autotuner:
    def __init__(self, path: str | None = DEFAULT_CACHE, candidates=CANDIDATES, reps: int = 3):
        self.path = path
        self.candidates = tuple(candidates)
        self.reps = reps
        self.cache: dict[str, int] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)
        self.timings: dict[str, dict[int, float]] = {}

    def save(self):
        if not self.path:
            return
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def time_config(self, n: int, d: int, B: int, K: int) -> float:
        """Median ms of one train step on a representative shape (depth and
        batch rounded to their buckets, capped to keep tuning short)."""
        dd, bb = min(bucket(d), 64), min(bucket(B), 64)
        sim = Simulator(n, dd, bb, tile_bits=K)
        rng = np.random.default_rng(0)
        theta = torch.from_numpy(rng.uniform(0, 2 * np.pi, 3 * n * dd).astype(np.float32)).cuda()
        x = torch.from_numpy(workloads.draw_x(bb, n, 1)).cuda()
        sim.train_step(theta, x)
        torch.cuda.synchronize()
        times = []
        for _ in range(self.reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            sim.train_step(theta, x)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        return float(np.median(times))

    def choose(self, n: int, d: int, B: int) -> int:
        """Tile width for a circuit; 0 (library default) when n <= 12."""
        if n <= 12:
            return 0
        k = key(n, d, B)
        if k not in self.cache:
            t = {K: self.time_config(n, d, B, K) for K in self.candidates}
            self.timings[k] = t
            self.cache[k] = min(t, key=t.get)
            self.save()
        return int(self.cache[k])

    __call__ = choose
