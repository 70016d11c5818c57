"""Data parallelism over samples (one process per GPU).

Samples are independent, so a batch is split into contiguous shards, one per
rank; each rank runs the fused train step on its shard and the only exchange
is the sum of the float64 gradient over ranks (the gradient of the total
loss). The paper suggests this for scaling out (DistributedDataParallel over
samples); no state is split across GPUs.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n_samples: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced [lo, hi) of rank's samples (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_samples, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def mean_weight(local: int, total: int) -> float:
    """Factor that turns the gradient of a local mean loss into this rank's
    share of the gradient of the global mean loss."""
    return local / total if total else 0.0


def allreduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum over ranks (no-op on a single process)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def dp_train_step(sim, theta, x_local, y_local, loss: str, n_total: int, group=None):
    """One data-parallel step: local fused train step, then the gradient (and
    loss) summed over ranks. For the mean-squared error the local gradient is
    weighted by local/total samples first."""
    lv, E, g = sim.train_step(theta, x_local, y_local, loss=loss)
    if loss == "mse":
        w = mean_weight(x_local.shape[0], n_total)
        g.mul_(w)
        lv.mul_(w)
    allreduce_sum(g, group)
    allreduce_sum(lv, group)
    return lv, E, g
