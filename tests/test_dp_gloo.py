"""Data-parallel path on CPU: two gloo ranks each train on their shard and
the summed gradient equals the single-process full-batch gradient.

The per-rank step here is a stand-in object whose train_step evaluates the
oracle (no GPU on this host); the sharding, loss weighting and all-reduce
under test are the library's (paper_2603_02804_gb300.dp).
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2603_02804_gb300 import dp, workloads

N, D, B = 6, 3, 10


class OracleStep:
    """train_step(theta, x, y, loss) with the float64 oracle, returning torch tensors."""

    def __init__(self, n, d):
        self.c = orc.hea(n, d)

    def train_step(self, theta, x, y=None, loss="sum"):
        th, xx = theta.double().numpy(), x.double().numpy()
        E = orc.expectation(self.c, th, xx, "Z", threads=1)
        if loss == "mse":
            yy = y.double().numpy()
            dLdE = orc.mse_dLdE(E, yy)
            lv = orc.mse_loss(E, yy)
        else:
            dLdE = np.ones(len(E))
            lv = float(E.sum())
        g, _ = orc.gradient(self.c, th, xx, "Z", dLdE=dLdE, threads=1)
        return torch.tensor([lv], dtype=torch.float64), torch.from_numpy(E), torch.from_numpy(g)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, loss, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = workloads.Workload("dp", N, D, B, loss, "Z", (11, 12, 13))
        theta, x, y = workloads.make_inputs(w)
        lo, hi = dp.shard_range(B, rank, world)
        sim = OracleStep(N, D)
        lv, _, g = dp.dp_train_step(sim, torch.from_numpy(theta), torch.from_numpy(x[lo:hi]),
                                    None if y is None else torch.from_numpy(y[lo:hi]), loss, B)
        q.put((rank, lv.item(), g.numpy()))
    finally:
        dist.destroy_process_group()


def test_shard_range_covers_every_sample_once():
    for n in (0, 1, 7, 10, 33):
        for world in (1, 2, 3, 4):
            ranges = [dp.shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, _) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("loss", ["sum", "mse"])
def test_two_gloo_ranks_sum_to_full_batch(loss):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, loss, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = workloads.Workload("dp", N, D, B, loss, "Z", (11, 12, 13))
    theta, x, y = workloads.make_inputs(w)
    lv, _, g = OracleStep(N, D).train_step(torch.from_numpy(theta), torch.from_numpy(x),
                                           None if y is None else torch.from_numpy(y), loss)
    for _, l_r, g_r in res:
        assert abs(l_r - lv.item()) < 1e-12
        assert np.max(np.abs(g_r - g.numpy())) < 1e-12
