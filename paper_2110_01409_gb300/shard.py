"""Column shards of the batched solves over ranks, one GPU each: the batched
form's multi-GPU path. Its B columns are independent problems (teleport
vectors or sources), so rank r solves a contiguous slice of them on its own
copy of the graph, and the only exchange is one gather of the result columns
at the end. Nothing crosses ranks during the sweeps.

Ranks come from torch.distributed when a process group is initialised (one
process per GPU, as torchrun starts them); without one there is a single rank
and nothing is exchanged.
"""
from __future__ import annotations

import torch


def column_range(B: int, world: int, rank: int) -> tuple[int, int]:
    """The slice [lo, hi) of B columns that rank solves: contiguous, in rank
    order, covering all B, slice sizes differing by at most one."""
    if B < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError(f"column_range({B}, {world}, {rank})")
    base, extra = divmod(B, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _ranks(group=None) -> tuple[int, int]:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def gather_columns(local: torch.Tensor, B: int, group=None) -> torch.Tensor:
    """Every rank's slice (local: [rows, hi - lo] of this rank's columns)
    assembled into [rows, B] on every rank, by one all_gather of slices padded
    to the widest."""
    rank, world = _ranks(group)
    if world == 1:
        return local
    import torch.distributed as dist

    rows = local.shape[0]
    width = -(-B // world)
    padded = torch.zeros((rows, width), dtype=local.dtype, device=local.device)
    padded[:, : local.shape[1]] = local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    out = torch.empty((rows, B), dtype=local.dtype, device=local.device)
    for r in range(world):
        lo, hi = column_range(B, world, r)
        out[:, lo:hi] = parts[r][:, : hi - lo]
    return out


def ppr_batched_sharded(plan, V: torch.Tensor, d=0.85, tol=1e-6, variant="async", delta=0, max_iters=1000,
                        group=None, solve=None):
    """Batched personalized PageRank with the columns of V [n, B] split over
    the ranks. Returns (R [n, B], iters [B]) on every rank. solve: the
    per-shard solver with the signature of dag.ppr_batched, which it is by
    default (a test passes a stand-in to check the sharding alone)."""
    if solve is None:
        from .dag import ppr_batched as solve
    rank, world = _ranks(group)
    n, B = V.shape
    lo, hi = column_range(B, world, rank)
    if hi > lo:
        R, iters, _ = solve(plan, V[:, lo:hi].contiguous(), d, tol, variant, delta, max_iters)
    else:
        R = torch.zeros((n, 0), dtype=V.dtype, device=V.device)
        iters = torch.zeros(0, dtype=torch.int32, device=V.device)
    return gather_columns(R, B, group), gather_columns(iters.view(1, -1), B, group).view(-1)


def sssp_batched_sharded(plan, srcs: torch.Tensor, w, variant="async", delta=0, max_iters=None, group=None,
                         solve=None):
    """Batched Bellman-Ford with the sources srcs [B] split over the ranks.
    Returns (D [n, B] int32 holding uint32 bits, iters [B]) on every rank.
    solve: the per-shard solver with the signature of dag.sssp_batched, which
    it is by default."""
    if solve is None:
        from .dag import sssp_batched as solve
    rank, world = _ranks(group)
    B = srcs.numel()
    lo, hi = column_range(B, world, rank)
    if hi > lo:
        D, iters, _ = solve(plan, srcs[lo:hi].contiguous(), w, variant, delta, max_iters)
        n = D.shape[0]
    else:
        n = int(plan.n)
        D = torch.zeros((n, 0), dtype=torch.int32, device=srcs.device)
        iters = torch.zeros(0, dtype=torch.int32, device=srcs.device)
    return gather_columns(D, B, group), gather_columns(iters.view(1, -1), B, group).view(-1)
