"""Data-parallel layout of the path and its one cross-process exchange.

Every matrix and every Monte Carlo walker is independent, so processes (one per
GPU) take contiguous slices of one seeded batch and exchange nothing while
they compute. The exchange comes at the end and is small: the per-order sums
of the connected sums of whole vertex sets (count, sum c, sum |c|, sum c^2 for
each order; the data of the power-series estimator of Section V, Eq. series),
reduced on each device by apm_order_sums and added across processes on host
tensors; and, when the surrogate network is trained data-parallel, its
gradient, averaged over the processes with each process's batch as weight
before every Adam step. Host tensors go through the initialised
torch.distributed process group (gloo); with no group, or one process, every
call is the identity.
"""
from __future__ import annotations

import math

import torch


def world() -> tuple[int, int]:
    """(rank, world size) of the initialised process group, else (0, 1)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard_bounds(total: int, rank: int, world_size: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous slice of `total` units; the first
    total % world_size ranks take one unit more."""
    if world_size < 1 or not 0 <= rank < world_size or total < 0:
        raise ValueError("need 0 <= rank < world_size and total >= 0")
    q, r = divmod(total, world_size)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def allreduce_sum_(t: torch.Tensor) -> torch.Tensor:
    """Sums a host tensor over the processes, in place."""
    import torch.distributed as dist
    if t.device.type != "cpu":
        raise TypeError("the exchange runs on host tensors")
    if world()[1] > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def combine_order_sums(local: torch.Tensor) -> torch.Tensor:
    """The per-order sums of all processes: `local` is this process's
    [n_max+1, 4] table (device or host, from apm_order_sums); returns the
    summed table as a float64 host tensor."""
    return allreduce_sum_(local.detach().to("cpu", torch.float64).contiguous().clone())


def estimator(sums: torch.Tensor) -> dict:
    """Per order m with samples: the mean of c_m, its standard error, the mean
    of |c_m| and the average sign sum c / sum |c|."""
    out = {}
    for m in range(sums.shape[0]):
        cnt, s1, sa, s2 = (float(v) for v in sums[m])
        if cnt < 1:
            continue
        mean = s1 / cnt
        var = max(s2 / cnt - mean * mean, 0.0)
        out[m] = {"count": int(round(cnt)), "mean": mean, "stderr": math.sqrt(var / max(cnt - 1.0, 1.0)),
                  "mean_abs": sa / cnt, "sign": s1 / sa if sa > 0 else 0.0}
    return out


def average_gradient_(grad: torch.Tensor, weight: float) -> torch.Tensor:
    """Replaces `grad` (device or host, float32) by the weighted average over the
    processes of their gradients, sum_r weight_r grad_r / sum_r weight_r. With
    each process's gradient the mean over its own rows and its row count as
    weight, the result is the gradient over the union of the rows."""
    if world()[1] == 1:
        return grad
    host = torch.empty(grad.numel() + 1, dtype=torch.float64)
    host[:-1] = grad.detach().reshape(-1).to("cpu", torch.float64) * float(weight)
    host[-1] = float(weight)
    allreduce_sum_(host)
    avg = (host[:-1] / host[-1]).to(torch.float32)
    grad.copy_(avg.reshape(grad.shape).to(grad.device))
    return grad
