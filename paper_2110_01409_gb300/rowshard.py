"""Row sharding of one synchronous solve across GPUs (one process per GPU).

The static partition of Sec. III-A, taken at GPU granularity, gives rank k
the contiguous rows [start[k], start[k+1]) balanced by in-degree + 1
(``dag.Plan.partition(world)``, every rank holding the whole graph in its own
plan). One synchronous sweep (Sec. I) is then:

1. every rank computes its rows from the whole previous iterate
   (``dag_pagerank_sweep_rows`` / ``dag_sssp_sweep_rows``, a warp-worker sweep
   of the row range);
2. an all-gather of the new row ranges (padded to the longest range) gives
   every rank the whole new iterate;
3. an all-reduce (sum) of the two FP64 per-range sums gives every rank the
   global residual (PageRank: L1 change; Bellman-Ford: rows lowered) and the
   mass on vertices with out-edges that the next sweep's dangling term needs.

Every rank applies the stopping rule of Sec. IV to the same global residual,
so all stop after the same sweep with the same iterate, which is the
unsharded synchronous iterate (same rows, same arithmetic per row).

The exchange logic here does not depend on the device: ``sweep`` is a
callable, the GPU one built by ``gpu_pagerank_sweep`` / ``gpu_sssp_sweep``,
and the tests run it with two ``gloo`` ranks on the CPU with the oracle's row
sweep standing in.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_ranges(starts) -> list[tuple[int, int]]:
    """(lo, hi) of every rank from the partition's block starts (world + 1 values)."""
    s = [int(x) for x in starts]
    return [(s[k], s[k + 1]) for k in range(len(s) - 1)]


def gather_ranges(local: torch.Tensor, ranges, full: torch.Tensor, group=None) -> torch.Tensor:
    """Writes every rank's row range into `full` (every rank's copy): an all-gather of the ranges,
    each padded to the longest. `local` holds this rank's range."""
    world = len(ranges)
    if world == 1:
        lo, hi = ranges[0]
        full[lo:hi] = local
        return full
    width = max(hi - lo for lo, hi in ranges)
    buf = torch.zeros(width, dtype=local.dtype, device=local.device)
    buf[: local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    for (lo, hi), part in zip(ranges, parts):
        full[lo:hi] = part[: hi - lo]
    return full


def reduce_sums(sums: torch.Tensor, world: int, group=None) -> torch.Tensor:
    """Sum of the per-range FP64 sums over the ranks (in place)."""
    if world > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums


def pagerank_sharded(sweep, x0: torch.Tensor, linked0: float, ranges, rank: int, tol: float = 1e-6,
                     max_iters: int = 1000, group=None):
    """Synchronous PageRank over row ranges. sweep(x_in, linked, x_out) writes this rank's range of
    x_out and returns its (residual, linked mass) sums as a float64 tensor [2]. Returns
    (x, sweeps, converged); every rank ends with the same whole iterate x."""
    world = len(ranges)
    lo, hi = ranges[rank]
    x, nxt = x0.clone(), x0.clone()
    linked = float(linked0)
    for it in range(1, max_iters + 1):
        sums = sweep(x, linked, nxt)
        gather_ranges(nxt[lo:hi].clone(), ranges, nxt, group)
        res, linked = (float(v) for v in reduce_sums(sums, world, group).cpu())
        x, nxt = nxt, x
        if res <= tol:
            return x, it, True
    return x, max_iters, False


def sssp_sharded(sweep, d0: torch.Tensor, ranges, rank: int, max_iters: int, group=None):
    """Synchronous Bellman-Ford over row ranges; sweep(d_in, d_out) returns the range's (rows lowered,
    0) sums. Stops after a sweep that lowered no row anywhere. Returns (dist, sweeps, converged)."""
    world = len(ranges)
    lo, hi = ranges[rank]
    d, nxt = d0.clone(), d0.clone()
    for it in range(1, max_iters + 1):
        sums = sweep(d, nxt)
        gather_ranges(nxt[lo:hi].clone(), ranges, nxt, group)
        changed = float(reduce_sums(sums, world, group)[0])
        d, nxt = nxt, d
        if changed == 0.0:
            return d, it, True
    return d, max_iters, False


def gpu_pagerank_sweep(dag, plan, lo: int, hi: int, d: float = 0.85, teleport=None, teleport_total: float = 1.0):
    """The GPU sweep of rows [lo, hi) for pagerank_sharded (state form x, see dag.rank_to_state)."""
    sums = torch.zeros(2, dtype=torch.float64, device=plan.rowptr.device)

    def sweep(x_in, linked, x_out):
        dag.pagerank_sweep_rows(plan, lo, hi, x_in, x_out, sums, d=d, teleport=teleport,
                                teleport_total=teleport_total, linked_mass=linked)
        return sums.clone()

    return sweep


def gpu_sssp_sweep(dag, plan, lo: int, hi: int, w8):
    """The GPU sweep of rows [lo, hi) for sssp_sharded (one-byte weights)."""
    sums = torch.zeros(2, dtype=torch.float64, device=plan.rowptr.device)

    def sweep(d_in, d_out):
        dag.sssp_sweep_rows(plan, lo, hi, w8, d_in, d_out, sums)
        return sums.clone()

    return sweep


def pagerank_row_sharded(dag, plan, rank: int, world: int, d: float = 0.85, tol: float = 1e-6,
                         max_iters: int = 1000, group=None) -> tuple[torch.Tensor, int, bool]:
    """PageRank (uniform teleport) of the plan's graph, rows split over `world` ranks as Sec. III-A
    splits them over workers. Returns (r, sweeps, converged), r the whole vector on every rank."""
    dev = plan.rowptr.device
    ranges = rank_ranges(plan.partition(world))
    lo, hi = ranges[rank]
    r0 = torch.full((plan.n,), 1.0 / plan.n, dtype=torch.float32, device=dev)
    x0 = torch.empty_like(r0)
    linked = torch.zeros(1, dtype=torch.float64, device=dev)
    dag.rank_to_state(plan, r0, x0, linked)
    x, it, ok = pagerank_sharded(gpu_pagerank_sweep(dag, plan, lo, hi, d), x0, float(linked.item()), ranges, rank,
                                 tol, max_iters, group)
    r = torch.empty_like(r0)
    dag.state_to_rank(plan, x, r)
    return r, it, ok


def sssp_row_sharded(dag, plan, src: int, w8, rank: int, world: int, group=None):
    """Bellman-Ford from src, rows split over `world` ranks. Returns (dist int32 holding uint32 bits,
    sweeps, converged) on every rank."""
    dev = plan.rowptr.device
    ranges = rank_ranges(plan.partition(world))
    lo, hi = ranges[rank]
    d0 = torch.full((plan.n,), -1, dtype=torch.int32, device=dev)  # 0xFFFFFFFF: unreachable
    d0[src] = 0
    return sssp_sharded(gpu_sssp_sweep(dag, plan, lo, hi, w8), d0, ranges, rank, plan.n + 1, group)
