"""Multi-GPU use of the solver: illumination angles are independent problems.

Each rank owns a contiguous share of the angles, runs its own solver handle on its own GPU, and
the only exchange is the sum of the per-rank data-term gradients (and losses) when the ranks
together form one inverse problem.  Without such a shared problem, ranks are plain replicas.
"""
from __future__ import annotations

from typing import Tuple

import torch


def shard(n: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of rank's contiguous share of n items (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_sum_(t: torch.Tensor) -> torch.Tensor:
    """In-place sum over all ranks of the default process group (no-op without one)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def sharded_loss_and_gradient(solver, f_d: torch.Tensor, theta_all: torch.Tensor, rec: torch.Tensor,
                              y_all: torch.Tensor, rank: int, world: int):
    """Loss 1/2 sum_q ||S u_q - y_q||^2 and its gradient in f_d over all angles, each rank solving
    its own share of the angles; one all-reduce of (loss, gradient)."""
    a, b = shard(theta_all.numel(), rank, world)
    solver.set_contrast(f_d)
    u, _ = solver.forward(theta_all[a:b])
    _, G, loss = solver.misfit(u, y_all[a:b], rec)
    g, _ = solver.gradient(theta_all[a:b], u, G)
    packed = torch.cat([torch.tensor([loss], dtype=torch.float64, device=g.device), g.reshape(-1)])
    allreduce_sum_(packed)
    return float(packed[0].item()), packed[1:].reshape(g.shape)
