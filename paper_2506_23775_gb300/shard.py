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


def exchange(part, group=None) -> np.ndarray:
    """All-gather one packed partial per rank and return their rank-order sum.

    ``part`` is a 1-D float64 tensor of the same length on every rank: on the
    current CUDA device for NCCL (the gather stays on the devices; only the
    gathered rows come to the host for the sum), on the CPU for gloo.  The sum
    runs on the host in rank order, so every rank gets the same bits.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    part = part.contiguous()
    if dist.get_backend(group) == "nccl":
        out = torch.empty((world,) + tuple(part.shape), dtype=part.dtype, device=part.device)
        dist.all_gather_into_tensor(out, part, group=group)
        return sum_in_rank_order(out.cpu().numpy())
    part = part.cpu()          # gloo gathers host tensors, one per rank
    bufs = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(bufs, part, group=group)
    return sum_in_rank_order(np.stack([b.numpy() for b in bufs]))


def sharded_eval(evaluate: Callable[[int, int], Tuple[float, np.ndarray, Optional[np.ndarray]]],
                 n_cols: int, n_params: int, k: int, group=None):
    """Evaluate this rank's shard with ``evaluate(c0, c1)`` and return the total.

    ``evaluate`` returns ``(f, rgrad, hvps)`` for the columns ``[c0, c1)`` (for
    example a device context restricted with ``rq_set_columns``).  The
    exchange is one all-gather of the packed partials over
    ``torch.distributed`` (gloo or NCCL); the sum is in rank order.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    c0, c1 = column_shard(n_cols, rank, world)
    part = torch.from_numpy(pack(*evaluate(c0, c1)))
    if dist.get_backend(group) == "nccl":
        part = part.to(torch.device("cuda", torch.cuda.current_device()))
    return unpack(exchange(part, group), n_params, k)


class DeviceShard:
    """Device-resident partials of one rank for the device-pointer entry points.

    ``buf`` is one float64 CUDA tensor laid out as ``[f, pad, rgrad, hvps]``
    (complex outputs 16-byte aligned, as the library requires), so that
    ``rq_hvp_dev`` writes this rank's partial straight into the buffer that
    the all-gather sends; ``total()`` exchanges it and returns
    ``(f, rgrad, hvps)`` summed in rank order.
    """

    def __init__(self, ctx, n_params: int, k: int, device):
        import torch
        self.ctx, self.P, self.k = ctx, n_params, k
        self.buf = torch.zeros(2 + 32 * n_params * (1 + k), dtype=torch.float64, device=device)
        base = self.buf.data_ptr()
        self.f_ptr = base
        self.g_ptr = base + 16
        self.h_ptr = base + 16 + 8 * 32 * n_params

    def evaluate(self, gates_ptr: int, dirs_ptr: int):
        """This rank's partial over the context's column range (stream-ordered)."""
        self.ctx.hvp_dev(gates_ptr, dirs_ptr, self.k, self.f_ptr, self.g_ptr, self.h_ptr)

    def total(self, stream=None, group=None):
        import torch
        if stream is not None:
            torch.cuda.current_stream().wait_stream(stream)
        v = exchange(self.buf, group)
        gsz = 32 * self.P
        f = float(v[0])
        rg = v[2:2 + gsz].copy().view(np.complex128).reshape(self.P, 4, 4)
        hv = v[2 + gsz:2 + gsz * (1 + self.k)].copy().view(np.complex128).reshape(self.k, self.P, 4, 4)
        return f, rg, hv


def context_evaluator(ctx, gates, dirs):
    """``evaluate(c0, c1)`` for a device context (``rq.Context``)."""
    def evaluate(c0: int, c1: int):
        ctx.set_columns(c0, c1)
        if dirs is None or len(dirs) == 0:
            f, g = ctx.grad(gates)
            return f, g, None
        return ctx.hvp(gates, dirs)
    return evaluate
