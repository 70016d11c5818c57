"""Autotuner for the fused path's plan options.

What it tunes, per (GPU, SM count, launch kind, n, depth bucket, batch
bucket), by timing qf_train_step (or the persistent batch step) on synthetic
inputs of that shape (depth and batch rounded up to powers of two, capped at
64; persistent batches are timed at 16 samples):

- tile width K (qubits held in shared memory per pass; fusion width of the
  pass, Sec. 3.2): 7..12 for circuits wider than one tile. A register group
  is always 4 qubits (16 amplitudes per thread), so K sets how many groups a
  pass visits and how many passes stream the state.
- catch-up rule of the round planner (strict or rising), for multi-tile
  round programs (the planner otherwise prices both on a prefix).
- forward kernel instance (2 or 3 CTAs per SM), single-circuit launches only.

The search is coordinate descent from the library defaults: the width first,
then the rule at the best width, then the instance. Results are cached in a
JSON file (or in memory). Circuits of at most 12 qubits hold the whole state
in one tile and keep the defaults.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "qfuse", "autotune.json")
WIDTHS = (11, 10, 9, 8, 7)   # and 12, the default for n > 12
RULES = (1, 2)          # catch_up: strict, rising
FWD_CTAS = (2, 3)
DEFAULT = {"tile_bits": 0, "catch_up": 0, "fwd_ctas": 0}


def bucket(v: int) -> int:
    """Power-of-two bucket (1, 2, 4, ...)."""
    return 1 << max(0, math.ceil(math.log2(max(1, v))))


def device_info() -> tuple[str, int]:
    """(name, SM count) of the current CUDA device."""
    import torch
    if not torch.cuda.is_available():
        return "cpu", 0
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return p.name, int(p.multi_processor_count)


def key(n: int, d: int, B: int, kind: str = "single", dev: tuple[str, int] | None = None) -> str:
    name, sms = dev if dev is not None else device_info()
    return f"{name}|sms={sms}|{kind}|n={n}|d~{d}|B~{B}"


# Persistent batches run many circuits' samples side by side, so the batch of
# one circuit does not change how its passes fill the GPU: batch-kind shapes
# are timed at this batch.
BATCH_KIND_SAMPLES = 16


def _synthetic(n, d, B, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    theta = torch.from_numpy(rng.uniform(0, 2 * np.pi, 3 * n * d).astype(np.float32)).cuda()
    x = torch.from_numpy(rng.uniform(0, np.pi, (B, n)).astype(np.float32)).cuda()
    return theta, x


def gpu_timer(n: int, d: int, B: int, cfg: dict, kind: str, reps: int = 3) -> float:
    """Median ms of one training step of an n-qubit, d-layer ansatz on B
    samples planned with cfg; kind "single" times qf_train_step, "batch" the
    persistent launch of that circuit alone."""
    import torch
    from .torch_api import Batch, Simulator
    theta, x = _synthetic(n, d, B)
    if kind == "batch":
        bt = Batch([(n, d, B)], loss="sum", tile_bits=lambda *_: dict(cfg))
        run = lambda: bt.train_step(theta, x)
    else:
        sim = Simulator(n, d, B, **cfg)
        run = lambda: sim.train_step(theta, x)
    run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return float(np.median(times))


class Autotuner:
    """Chooses plan options per circuit shape; `choose(n, d, B)` returns a
    dict of qf_plan options (tile_bits, catch_up, fwd_ctas).

    timer(n, d, B, cfg, kind) -> ms may be replaced (tests pass a model);
    dev = (name, SM count) overrides the device the cache keys name."""

    def __init__(self, path: str | None = DEFAULT_CACHE, kind: str = "single", timer=None, dev=None,
                 max_depth: int = 64, max_batch: int = 64):
        self.path = path
        self.kind = kind
        self.timer = timer or gpu_timer
        self.dev = dev
        self.max_depth, self.max_batch = max_depth, max_batch
        self.cache: dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)
        self.timings: dict[str, dict[str, float]] = {}
        self.trials = 0

    def save(self):
        if not self.path:
            return
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def _time(self, n, d, B, cfg, log):
        tag = json.dumps(cfg, sort_keys=True)
        if tag not in log:
            self.trials += 1
            try:
                log[tag] = float(self.timer(n, d, B, cfg, self.kind))
            except Exception:  # a configuration the planner refuses
                log[tag] = float("inf")
        return log[tag]

    def shape(self, n: int, d: int, B: int) -> tuple[int, int, int]:
        """The shape timed for a circuit: depth and batch rounded up to powers
        of two and capped (a batch-kind tuner times every batch at 16)."""
        bb = BATCH_KIND_SAMPLES if self.kind == "batch" else min(bucket(B), self.max_batch)
        return n, min(bucket(d), self.max_depth), bb

    def search(self, n: int, d: int, B: int) -> tuple[dict, dict]:
        """Coordinate descent over width, rule and instance on the timed
        shape."""
        _, dd, bb = self.shape(n, d, B)
        log: dict[str, float] = {}
        best = dict(DEFAULT)
        best_t = self._time(n, dd, bb, best, log)
        for K in WIDTHS:
            if K >= n:
                continue
            cfg = dict(best, tile_bits=K)
            t = self._time(n, dd, bb, cfg, log)
            if t < best_t:
                best, best_t = cfg, t
        for r in RULES:
            cfg = dict(best, catch_up=r)
            t = self._time(n, dd, bb, cfg, log)
            if t < best_t:
                best, best_t = cfg, t
        if self.kind == "single":
            for f in FWD_CTAS:
                cfg = dict(best, fwd_ctas=f)
                t = self._time(n, dd, bb, cfg, log)
                if t < best_t:
                    best, best_t = cfg, t
        return best, log

    def choose(self, n: int, d: int, B: int) -> dict:
        """Plan options for a circuit (the defaults when n <= 12)."""
        if n <= 12:
            return dict(DEFAULT)
        k = key(*self.shape(n, d, B), self.kind, self.dev)
        if k not in self.cache:
            best, log = self.search(n, d, B)
            self.timings[k] = log
            self.cache[k] = best
            self.save()
        return dict(self.cache[k])

    __call__ = choose
