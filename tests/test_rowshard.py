"""Row sharding across ranks (rowshard.py) on the CPU: two gloo ranks, each
computing its row range of every synchronous sweep with the oracle's row sweep
standing in for the GPU, exchange by all-gather and all-reduce. Every rank
must end with the unsharded oracle's synchronous iterate (PageRank: same
sweeps, L1 within FP64 rounding; Bellman-Ford: the same distances and sweep
count), for an uneven split, an empty range and a single rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import paper_2110_01409_gb300.inputs as I
from paper_2110_01409_gb300 import rowshard as RS


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pr_sweep(g, lo, hi):
    def sweep(x_in, linked, x_out):
        out = x_out.numpy()
        res, lk = oracle.pagerank_sweep_rows(g, lo, hi, x_in.numpy(), out, N=linked)
        return torch.tensor([res, lk], dtype=torch.float64)
    return sweep


def _bf_sweep(g, w, lo, hi):
    def sweep(d_in, d_out):
        c = oracle.sssp_sweep_rows(g, w, lo, hi, d_in.numpy().view(np.uint32), d_out.numpy().view(np.uint32))
        return torch.tensor([float(c), 0.0], dtype=torch.float64)
    return sweep


def _worker(rank, world, port, starts, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = I.rmat(11, 16, seed=5)
        w = I.weights_u32(g, 5)
        ranges = RS.rank_ranges(starts)
        lo, hi = ranges[rank]
        r0 = np.full(g.n, 1.0 / g.n)
        od = np.bincount(g.colidx, minlength=g.n)
        x, it, ok = RS.pagerank_sharded(_pr_sweep(g, lo, hi), torch.from_numpy(r0.copy()), float(r0[od > 0].sum()),
                                        ranges, rank, tol=1e-6, max_iters=500)
        d0 = np.full(g.n, oracle.INF, dtype=np.uint32)
        d0[3] = 0
        dd, it2, ok2 = RS.sssp_sharded(_bf_sweep(g, w, lo, hi), torch.from_numpy(d0.view(np.int32).copy()), ranges,
                                       rank, g.n + 1)
        q.put((rank, x.numpy(), it, ok, dd.numpy().view(np.uint32).copy(), it2, ok2))
    finally:
        dist.destroy_process_group()


def _run(starts, world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, starts, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda t: t[0])


@pytest.mark.parametrize("starts_kind", ["balanced", "uneven", "empty"])
def test_two_gloo_ranks_equal_the_unsharded_sync_solve(starts_kind):
    g = I.rmat(11, 16, seed=5)
    w = I.weights_u32(g, 5)
    if starts_kind == "balanced":
        starts = oracle.partition(g, 2)  # Sec. III-A at rank granularity
    elif starts_kind == "uneven":
        starts = np.array([0, 100, g.n])
    else:
        starts = np.array([0, g.n, g.n])  # rank 1 owns no row
    res = _run([int(s) for s in starts], 2)
    r_ref, it_ref, _, _ = oracle.pagerank(g, oracle.SYNC, tol=1e-6)
    d_ref, it2_ref, _, _ = oracle.sssp(g, w, 3, oracle.SYNC)
    for rank, x, it, ok, dd, it2, ok2 in res:
        assert ok and it == it_ref, (rank, it, it_ref)
        assert np.abs(x - r_ref).sum() <= 1e-12
        assert ok2 and it2 == it2_ref and np.array_equal(dd, d_ref)


def test_single_rank_needs_no_collective():
    g = I.rmat(9, 16, seed=2)
    r0 = np.full(g.n, 1.0 / g.n)
    od = np.bincount(g.colidx, minlength=g.n)
    x, it, ok = RS.pagerank_sharded(_pr_sweep(g, 0, g.n), torch.from_numpy(r0.copy()), float(r0[od > 0].sum()),
                                    [(0, g.n)], 0, tol=1e-6, max_iters=500)
    r_ref, it_ref, _, _ = oracle.pagerank(g, oracle.SYNC, tol=1e-6)
    assert ok and it == it_ref and np.abs(x.numpy() - r_ref).sum() <= 1e-12


def test_rank_ranges_from_partition_starts():
    assert RS.rank_ranges([0, 5, 5, 9]) == [(0, 5), (5, 5), (5, 9)]
