"""The core phase (Algorithm 5) over a training set split across processes.

Algorithm 5's core gradient G^(n) = sum_Omega (xhat - x) a^(n)T d^(n) is a sum
over the nonzeros, computed from one fixed A and B, so it splits over any
partition of Omega.  Each process keeps a context over one contiguous shard
of the nonzeros (``shard_range``) and computes its shard's gradient
(``ft_core_grad``); one all-reduce adds the shards' gradients (sum_n J_n R
floats: 768 at N = 3, J = R = 16); every process then applies the same step
with |Omega| = the total number of nonzeros (``ft_core_apply``), so B stays
identical everywhere.  The sum is what the single-process core phase computes,
up to the order of the float32 additions across shards.

The factor phase is not split this way: rows are shared by nonzeros of every
shard and the Hogwild pass needs one shared A.  These helpers only marshal
arguments and call the collective; every arithmetic step runs in the CUDA
library (the gradient and the step) or in the collective (the sum).
"""
from __future__ import annotations

import contextlib

import torch
import torch.distributed as dist

from . import ft


def shard_range(nnz: int, rank: int, world: int) -> tuple[int, int]:
    """The nonzeros [lo, hi) of shard ``rank`` of ``world``: contiguous
    ranges in stored order whose sizes differ by at most one and which cover
    [0, nnz) once, in rank order (empty shards when nnz < world)."""
    if world < 1 or not 0 <= rank < world or nnz < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and nnz >= 0")
    return nnz * rank // world, nnz * (rank + 1) // world


def allreduce_core_grad(G: torch.Tensor, group=None) -> torch.Tensor:
    """Sum ``G`` (the flat gradient of ``ft_core_grad``) in place over the
    ranks of ``group`` (the default group if None).  Without an initialised
    process group, or with one rank, G is left as it is."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(G, op=dist.ReduceOp.SUM, group=group)
    return G


def epoch_core_sharded(model: "ft.FastTuckerPlus", lr: float, lam: float, nnz_total: int,
                       group=None, stream=None) -> torch.Tensor:
    """One core phase of Algorithm 5 over all shards: this process's shard
    gradient (``model`` is a context over the shard), summed over the group,
    then the step B <- B - lr (G / nnz_total + lam B) on ``model``'s B.
    ``nnz_total`` is |Omega|, the sum of every shard's nnz.  ``stream``: None
    (torch's current stream) or a torch.cuda.Stream, on which the gradient,
    the collective and the step are ordered.  Returns the summed gradient
    (flat, the layout of ``ft_core_grad``)."""
    scope = torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()
    with scope:
        G = torch.empty(sum(j * model.R for j in model.J), dtype=torch.float32,
                        device=model.vals.device)
        ft.ft_core_grad(model.ctx, G)
        allreduce_core_grad(G, group)
        ft.ft_core_apply(model.ctx, G, nnz_total, lr, lam)
    return G
