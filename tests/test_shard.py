"""Column shards of the batched solves (the batched form's multi-GPU path):
rank r solves a contiguous slice of the columns and the only exchange is the
final gather. Two gloo ranks on the CPU, with the oracle standing in for each
rank's GPU solve, so that what is checked is the sharding itself: each rank
solves exactly its slice, and every rank ends with all columns in order, equal
to the unsharded oracle results."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import paper_2110_01409_gb300.inputs as I
from paper_2110_01409_gb300.shard import column_range, gather_columns, ppr_batched_sharded, sssp_batched_sharded


@pytest.mark.parametrize("B,world", [(0, 1), (1, 2), (5, 2), (7, 3), (256, 8), (3, 4)])
def test_column_range_covers_in_order_and_balances(B, world):
    ranges = [column_range(B, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == B
    for (lo, hi), (lo2, _) in zip(ranges, ranges[1:]):
        assert hi == lo2  # contiguous, rank order
    sizes = [hi - lo for lo, hi in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


def test_column_range_rejects_bad_ranks():
    for args in [(4, 2, 2), (4, 0, 0), (-1, 2, 0), (4, 2, -1)]:
        with pytest.raises(ValueError):
            column_range(*args)


def test_single_rank_needs_no_exchange():
    x = torch.arange(6, dtype=torch.float32).view(2, 3)
    assert gather_columns(x, 3) is x


def _graph():
    return I.rmat(8, 8, seed=3)


def _teleports(n, B):
    rng = np.random.default_rng(11)
    V = rng.random((n, B))
    return V / V.sum(axis=0)


def _oracle_ppr_shard(calls):
    def solve(g, Vs, d, tol, variant, delta, max_iters):
        calls.append(Vs.shape[1])
        cols = [oracle.pagerank(g, oracle.SYNC, d=d, tol=tol, tele=Vs[:, c].double().numpy())[0]
                for c in range(Vs.shape[1])]
        R = torch.from_numpy(np.stack(cols, axis=1).astype(np.float32))
        return R, torch.full((Vs.shape[1],), 7, dtype=torch.int32), None
    return solve


def _oracle_sssp_shard(calls):
    def solve(g, srcs, w, variant, delta, max_iters):
        calls.append(srcs.numel())
        cols = [oracle.dijkstra(g, w, int(s)) for s in srcs.tolist()]
        D = torch.from_numpy(np.stack(cols, axis=1).view(np.int32))
        return D, torch.full((srcs.numel(),), 5, dtype=torch.int32), None
    return solve


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, B_ppr, B_sssp, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = _graph()
        V = torch.from_numpy(_teleports(g.n, B_ppr).astype(np.float32))
        calls_p, calls_s = [], []
        R, it_p = ppr_batched_sharded(g, V, 0.85, 1e-9, solve=_oracle_ppr_shard(calls_p))
        w = I.weights_u32(g, 3)
        srcs = torch.from_numpy(I.sources(g, B_sssp, seed=3).astype(np.int32))
        D, it_s = sssp_batched_sharded(g, srcs, w, solve=_oracle_sssp_shard(calls_s))
        out[rank] = (R.numpy(), it_p.numpy(), D.numpy(), it_s.numpy(), calls_p, calls_s)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("B_ppr,B_sssp", [(5, 3), (1, 1)])
def test_two_ranks_solve_their_slices_and_all_get_every_column(B_ppr, B_sssp):
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, B_ppr, B_sssp, out), nprocs=world, start_method="spawn",
                           join=True)
        res = dict(out)
    g = _graph()
    V = _teleports(g.n, B_ppr).astype(np.float32)
    R_ref = np.stack([oracle.pagerank(g, oracle.SYNC, d=0.85, tol=1e-9, tele=V[:, c].astype(np.float64))[0]
                      for c in range(B_ppr)], axis=1).astype(np.float32)
    w = I.weights_u32(g, 3)
    srcs = I.sources(g, B_sssp, seed=3)
    D_ref = np.stack([oracle.dijkstra(g, w, int(s)) for s in srcs], axis=1).view(np.int32)
    for r in range(world):
        R, it_p, D, it_s, calls_p, calls_s = res[r]
        lo, hi = column_range(B_ppr, world, r)
        assert calls_p == ([hi - lo] if hi > lo else [])  # this rank solved its slice only
        lo, hi = column_range(B_sssp, world, r)
        assert calls_s == ([hi - lo] if hi > lo else [])
        assert np.array_equal(R, R_ref)  # every column, in order, on every rank
        assert np.array_equal(D, D_ref)
        assert list(it_p) == [7] * B_ppr and list(it_s) == [5] * B_sssp
