"""Column sharding of the basis sum across ranks (one process per GPU).

The basis sum of Eq. f_target_sum_unit_vec is embarrassingly parallel (paper
Sec. "Parallelization": OpenMP threads and MPI ranks over basis vectors).
Each rank evaluates a contiguous column range with its own device context;
the partial cost, Riemannian gradient and HVPs are exchanged once per
evaluation (1 + 32 * n_params * (1 + k) doubles) and summed in rank order on
every rank, so all ranks hold the same, reproducible total.  Every output is
linear in the per-column terms, so the partial sums add up exactly (up to the
rounding of the sum order).
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import numpy as np


def column_shard(n_cols: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous, balanced column range of ``rank`` out of ``world``."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return (rank * n_cols) // world, ((rank + 1) * n_cols) // world


def pack(f: float, rgrad: np.ndarray, hvps: Optional[np.ndarray]) -> np.ndarray:
    parts = [np.array([f], dtype=np.float64), np.ascontiguousarray(rgrad).view(np.float64).ravel()]
    if hvps is not None:
        parts.append(np.ascontiguousarray(hvps).view(np.float64).ravel())
    return np.concatenate(parts)


def unpack(v: np.ndarray, n_params: int, k: int):
    gsz = n_params * 32
    f = float(v[0])
    rg = v[1:1 + gsz].copy().view(np.complex128).reshape(n_params, 4, 4)
    hv = v[1 + gsz:1 + gsz * (1 + k)].copy().view(np.complex128).reshape(k, n_params, 4, 4) if k else None
    return f, rg, hv


def sum_in_rank_order(stack: np.ndarray) -> np.ndarray:
    """Fixed-order sum of the per-rank rows (rank 0 first)."""
    out = stack[0].copy()
    for r in range(1, stack.shape[0]):
        out += stack[r]
    return out


def sharded_eval(evaluate: Callable[[int, int], Tuple[float, np.ndarray, Optional[np.ndarray]]],
                 n_cols: int, n_params: int, k: int, group=None):
    """Evaluate this rank's shard with ``evaluate(c0, c1)`` and return the total.

    ``evaluate`` returns ``(f, rgrad, hvps)`` for the columns ``[c0, c1)`` (for
    example a device context restricted with ``rq_set_columns``).  The
    exchange is one ``all_gather`` of the packed partials over
    ``torch.distributed`` (gloo or NCCL); the sum is in rank order.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    c0, c1 = column_shard(n_cols, rank, world)
    part = pack(*evaluate(c0, c1))
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.from_numpy(part).to(dev)
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t, group=group)
    stack = np.stack([b.cpu().numpy() for b in bufs])
    return unpack(sum_in_rank_order(stack), n_params, k)


def context_evaluator(ctx, gates, dirs):
    """``evaluate(c0, c1)`` for a device context (``rq.Context``)."""
    def evaluate(c0: int, c1: int):
        ctx.set_columns(c0, c1)
        if dirs is None or len(dirs) == 0:
            f, g = ctx.grad(gates)
            return f, g, None
        return ctx.hvp(gates, dirs)
    return evaluate
