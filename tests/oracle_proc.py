"""Oracle calls in a spawned worker process, for the large cases of the GPU
tests.

A test process that has loaded torch and created a CUDA context also holds
their worker threads. The oracle's OpenMP threads, started in that process,
contend with them for the host cores, and the oracle then runs several times
slower than in a clean process. The worker is started with the spawn method,
so it inherits no CUDA state and loads no torch, and its OpenMP threads leave
two cores free. It runs the oracle module's functions unchanged.
"""
from __future__ import annotations

import atexit
import multiprocessing as mp
import os

_pool = None


def _init():
    # leave two host cores to the test process and the driver's threads
    os.environ.setdefault("OMP_NUM_THREADS", str(max(1, (os.cpu_count() or 1) - 2)))


def _call(name, args, kwargs):
    from oracle import oracle as orc
    return getattr(orc, name)(*args, **kwargs)


def _close():
    global _pool
    if _pool is not None:
        _pool.terminate()
        _pool.join()
        _pool = None


def call(name: str, *args, **kwargs):
    """oracle.<name>(*args, **kwargs), evaluated in the worker process."""
    global _pool
    if _pool is None:
        _pool = mp.get_context("spawn").Pool(1, initializer=_init)
        atexit.register(_close)
    return _pool.apply(_call, (name, args, kwargs))
