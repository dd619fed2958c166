"""GPU parity of the frontier Bellman-Ford (tiles run only when an input changed).

Synchronous form: distances bit-exact against Dijkstra, the sweep count of the
plain synchronous oracle, and the edges the launch ran equal to the frontier
oracle's exact count for the same partition and tile size. Asynchronous form:
distances bit-exact, edges between one full sweep and sweeps * m.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import frontier
import paper_2110_01409_gb300.inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dag():
    from paper_2110_01409_gb300 import build, dag as D

    build.build()
    assert torch.cuda.is_available()
    return D


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _weights(g, seed, u8):
    w = I.weights_u32(g, seed)
    wd = torch.from_numpy(w.astype(np.uint8) if u8 else w.view(np.int32)).cuda()
    return w, wd


GRAPHS = [lambda: I.rmat(13, 16, seed=2), lambda: I.rmat(14, 8, seed=5),
          lambda: I.banded(30011, 15, 1024, 1, seed=3), lambda: I.erdos_renyi(20000, 8, seed=4)]


@pytest.mark.parametrize("maker", GRAPHS)
@pytest.mark.parametrize("u8", [True, False])
def test_sync_frontier_exact_edges(dag, maker, u8):
    g = maker()
    w, wd = _weights(g, 1, u8)
    src = int(I.sources(g, 1, seed=3)[0])
    plan = dag.Plan.from_graph(g, "cuda")
    d, st = dag.sssp(plan, src, wd, "sync", 0, reads="frontier")
    assert st["converged"]
    assert np.array_equal(_u32(d), oracle.dijkstra(g, w, src))
    start = oracle.partition(g, st["workers"])
    d_o, it_o, ed_o, ok = frontier.sssp_frontier_sync(g, w, src, start, dag.tile_items())
    _, it_sync, _, _ = oracle.sssp(g, w, src, oracle.SYNC)
    assert ok and it_o == it_sync and st["iters"] == it_sync
    assert st["edges_processed"] == int(ed_o.sum()), (st["edges_processed"], int(ed_o.sum()), g.m * it_sync)


@pytest.mark.parametrize("maker", GRAPHS)
@pytest.mark.parametrize("reads", ["frontier", "own_l1+frontier", "cached+frontier"])
def test_async_frontier_exact_distances(dag, maker, reads):
    g = maker()
    w, wd = _weights(g, 2, True)
    src = int(I.sources(g, 1, seed=4)[0])
    plan = dag.Plan.from_graph(g, "cuda")
    d, st = dag.sssp(plan, src, wd, "async", 0, reads=reads)
    assert st["converged"]
    assert np.array_equal(_u32(d), oracle.dijkstra(g, w, src))
    assert g.m <= st["edges_processed"] <= st["iters"] * g.m
    # the plain asynchronous solve on the same plan afterwards is unaffected
    d2, st2 = dag.sssp(plan, src, wd, "async", 0)
    assert np.array_equal(_u32(d2), _u32(d)) and st2["edges_processed"] == st2["iters"] * g.m


def test_frontier_skips_work_on_rmat(dag):
    g = I.rmat(16, 16, seed=2)
    w, wd = _weights(g, 1, True)
    src = int(I.sources(g, 1, seed=2)[0])
    plan = dag.Plan.from_graph(g, "cuda")
    _, st_plain = dag.sssp(plan, src, wd, "sync", 0)
    _, st = dag.sssp(plan, src, wd, "sync", 0, reads="frontier")
    assert st["iters"] == st_plain["iters"]
    assert st["edges_processed"] < 0.9 * st_plain["edges_processed"]


def test_frontier_edge_cases_and_rejections(dag):
    # isolated source: one sweep over everything, nothing changes
    g = I.from_edges(6, [0, 1, 2], [1, 2, 3], "tiny")
    w = np.array([5, 6, 7], dtype=np.uint32)
    plan = dag.Plan.from_graph(g, "cuda")
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    for var in ["sync", "async"]:
        d, st = dag.sssp(plan, 4, wd, var, 0, reads="frontier")
        assert list(_u32(d)) == [0xFFFFFFFF] * 4 + [0, 0xFFFFFFFF] and st["iters"] == 1
        assert st["edges_processed"] == g.m
        d, st = dag.sssp(plan, 0, wd, var, 0, reads="frontier")
        assert list(_u32(d)) == [0, 5, 11, 18, 0xFFFFFFFF, 0xFFFFFFFF]
    with pytest.raises(dag.DagError):
        dag.sssp(plan, 0, wd, "delayed", 16, reads="frontier")
    with pytest.raises(dag.DagError):
        dag.pagerank(plan, 0.85, 1e-6, "async", 0, reads="frontier")


# ---- the warp-tile frontier (DAG_WARP_WORKERS | DAG_SSSP_FRONTIER, asynchronous form) ----
WARP_READS = ["warp+frontier", "warp+cached+frontier", "ordered+frontier", "ordered+cached+frontier"]


@pytest.mark.parametrize("maker", GRAPHS + [lambda: I.from_edges(200001, np.arange(1, 200001),
                                                                 np.zeros(200000, dtype=np.int64), "instar")])
@pytest.mark.parametrize("reads", WARP_READS)
def test_warp_frontier_exact_distances(dag, maker, reads):
    # distances bit-exact against Dijkstra; the edges run lie between one full sweep and a full sweep per
    # sweep; every value read is at most one sweep old, so no more sweeps than the synchronous form
    g = maker()
    w, wd = _weights(g, 2, True)
    src = int(I.sources(g, 1, seed=4)[0])
    plan = dag.Plan.from_graph(g, "cuda")
    for ipt in (5, 7, 11):
        plan.set_warp_tile(ipt)
        d, st = dag.sssp(plan, src, wd, "async", 0, reads=reads)
        assert st["converged"], st
        assert np.array_equal(_u32(d), oracle.dijkstra(g, w, src)), ipt
        assert g.m <= st["edges_processed"] <= st["iters"] * g.m
        _, it_sync, _, _ = oracle.sssp(g, w, src, oracle.SYNC)
        assert st["iters"] <= it_sync


@pytest.mark.parametrize("reads", WARP_READS)
def test_warp_frontier_thresholds(dag, reads):
    # 0 marks per tile keeps every sweep dense (every edge every sweep); a huge threshold makes every sweep
    # after the first sparse (fewer edges); both give Dijkstra's distances, four-byte weights too
    g = I.rmat(16, 16, seed=2)
    for u8 in (True, False):
        w, wd = _weights(g, 3, u8)
        src = int(I.sources(g, 1, seed=2)[0])
        ref = oracle.dijkstra(g, w, src)
        plan = dag.Plan.from_graph(g, "cuda")
        plan.set_warp_frontier_marks(0.0)
        d, st = dag.sssp(plan, src, wd, "async", 0, reads=reads)
        assert st["converged"] and np.array_equal(_u32(d), ref)
        assert st["edges_processed"] == st["iters"] * g.m
        plan.set_warp_frontier_marks(1e6)
        d, st = dag.sssp(plan, src, wd, "async", 0, reads=reads)
        assert st["converged"] and np.array_equal(_u32(d), ref)
        assert st["edges_processed"] < 0.9 * st["iters"] * g.m
        plan.set_warp_frontier_marks(1.0)
        d, st = dag.sssp(plan, src, wd, "async", 0, reads=reads)
        assert st["converged"] and np.array_equal(_u32(d), ref)
    with pytest.raises(dag.DagError):
        plan.set_warp_frontier_marks(-1.0)


def test_warp_frontier_edge_cases(dag):
    g = I.from_edges(6, [0, 1, 2], [1, 2, 3], "tiny")
    w = np.array([5, 6, 7], dtype=np.uint32)
    plan = dag.Plan.from_graph(g, "cuda")
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    for reads in WARP_READS:
        d, st = dag.sssp(plan, 4, wd, "async", 0, reads=reads)  # isolated source: one sweep, nothing changes
        assert list(_u32(d)) == [0xFFFFFFFF] * 4 + [0, 0xFFFFFFFF] and st["iters"] == 1
        d, st = dag.sssp(plan, 0, wd, "async", 0, reads=reads)
        assert list(_u32(d)) == [0, 5, 11, 18, 0xFFFFFFFF, 0xFFFFFFFF]
    empty = I.from_edges(5, [], [], "empty")
    pe = dag.Plan.from_graph(empty, "cuda")
    d, st = dag.sssp(pe, 2, torch.zeros(1, dtype=torch.int32, device="cuda"), "async", 0, reads="warp+frontier")
    assert list(_u32(d)) == [0xFFFFFFFF, 0xFFFFFFFF, 0, 0xFFFFFFFF, 0xFFFFFFFF] and st["iters"] == 1


def test_warp_frontier_barrier_timeout_leaves_context_usable(dag):
    g = I.rmat(12, 16, seed=2)
    w, wd = _weights(g, 1, True)
    plan = dag.Plan.from_graph(g, "cuda")
    plan.debug_skip_barrier_once(100)
    with pytest.raises(dag.DagError) as ei:
        dag.sssp(plan, 3, wd, "async", 0, reads="warp+frontier")
    assert ei.value.code == dag.ERR_BARRIER_TIMEOUT
    d, st = dag.sssp(plan, 3, wd, "async", 0, reads="warp+frontier")
    assert st["converged"] and np.array_equal(_u32(d), oracle.dijkstra(g, w, 3))
