"""GPU parity of the batched PPR / SSSP launch against the CPU oracle (C ABI).

Each column of a batched solve is an independent problem: PPR columns must be
within L1 1e-5 of their fp64 fixed points (same bound as the single-vector
PageRank), SSSP columns bit-exact against Dijkstra, and in the synchronous form
each column must run exactly as many sweeps as its single-vector solve.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_01409_gb300.inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dag():
    from paper_2110_01409_gb300 import build, dag as D

    build.build()
    assert torch.cuda.is_available()
    return D


@pytest.fixture(scope="module")
def graph():
    return I.rmat(12, 16, seed=31)


@pytest.mark.parametrize("variant,delta", [("sync", 0), ("async", 0), ("delayed", 4), ("delayed", 16)])
def test_ppr_batched_columns_match_oracle(dag, graph, variant, delta):
    g = graph
    B = 40  # not a multiple of 32: a ragged last warp
    sets = I.ppr_seed_sets(g.n, B, seed=7)
    V = I.teleport_matrix(g.n, sets)
    plan = dag.Plan.from_graph(g, "cuda")
    R, iters, st = dag.ppr_batched(plan, torch.from_numpy(V).cuda(), 0.85, 1e-6, variant, delta)
    assert st["converged"], st
    R = R.cpu().numpy().astype(np.float64)
    its = iters.cpu().numpy()
    for c in [0, 1, 17, 31, 32, 39]:
        rstar = oracle.pagerank_fixed_point(g, 0.85, tele=V[:, c].astype(np.float64))
        assert np.abs(R[:, c] - rstar).sum() <= 1e-5, c
        if variant == "sync":
            _, st1 = dag.pagerank(plan, 0.85, 1e-6, "sync", 0, teleport=torch.from_numpy(V[:, c].copy()).cuda())
            assert abs(int(its[c]) - st1["iters"]) <= 1
    assert st["column_sweeps"] == int(its.sum())
    assert st["sweeps"] == int(its.max())


def test_ppr_batched_cycle_closed_form(dag):
    n, d = 256, 0.85
    g = I.from_edges(n, np.arange(n), (np.arange(n) + 1) % n)
    srcs = [0, 5, 77, 255]
    V = np.zeros((n, len(srcs)), dtype=np.float32)
    for c, s in enumerate(srcs):
        V[s, c] = 1.0
    plan = dag.Plan.from_graph(g, "cuda")
    R, _, st = dag.ppr_batched(plan, torch.from_numpy(V).cuda(), d, 1e-8, "delayed", 8)
    R = R.cpu().numpy()
    for c, s in enumerate(srcs):
        want = np.array([(1 - d) * d ** ((v - s) % n) / (1 - d ** n) for v in range(n)])
        assert np.max(np.abs(R[:, c] - want)) <= 1e-6


@pytest.mark.parametrize("variant,delta", [("sync", 0), ("async", 0), ("delayed", 8)])
def test_sssp_batched_bit_exact(dag, graph, variant, delta):
    g = graph
    w = I.weights_u32(g, 9)
    srcs = I.sources(g, 33, seed=5)
    plan = dag.Plan.from_graph(g, "cuda")
    D, iters, st = dag.sssp_batched(plan, torch.from_numpy(srcs.view(np.int32)).cuda(),
                                    torch.from_numpy(w.view(np.int32)).cuda(), variant, delta)
    assert st["converged"]
    D = D.cpu().numpy().view(np.uint32)
    its = iters.cpu().numpy()
    for c, s in enumerate(srcs):
        ref = oracle.dijkstra(g, w, int(s))
        assert np.array_equal(D[:, c], ref), c
        if variant == "sync":
            _, it, _, _ = oracle.sssp(g, w, int(s), oracle.SYNC)
            assert its[c] == it


def test_batched_single_column_and_bad_source(dag, graph):
    g = graph
    plan = dag.Plan.from_graph(g, "cuda")
    V = np.zeros((g.n, 1), dtype=np.float32)
    V[:, 0] = 1.0 / g.n
    R, iters, st = dag.ppr_batched(plan, torch.from_numpy(V).cuda(), 0.85, 1e-6, "delayed", 16)
    assert np.abs(R.cpu().numpy()[:, 0].astype(np.float64) - oracle.pagerank_fixed_point(g)).sum() <= 1e-5
    w = torch.from_numpy(I.weights_u32(g, 1).view(np.int32)).cuda()
    with pytest.raises(dag.DagError):
        dag.sssp_batched(plan, torch.tensor([0, g.n + 5], dtype=torch.int32, device="cuda"), w)
