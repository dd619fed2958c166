"""GPU row-range sweeps (dag_pagerank_sweep_rows / dag_sssp_sweep_rows) and the
row-sharded solve on one GPU: with one rank, and with the ranks' ranges run one
after the other in one process (the exchange is then the shared arrays), the
synchronous iterates must be the oracle's: PageRank within L1 1e-5 of the fp64
fixed point with the oracle's sync sweep count (+-1), Bellman-Ford bit-exact
with the same sweep count."""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_01409_gb300.inputs as I
from paper_2110_01409_gb300 import rowshard as RS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dag():
    from paper_2110_01409_gb300 import build, dag as D

    build.build()
    return D


GRAPHS = [lambda: I.rmat(14, 16, seed=5), lambda: I.banded(30011, 15, 1024, 1, seed=3),
          lambda: I.from_edges(200001, np.arange(1, 200001), np.zeros(200000, dtype=np.int64), name="instar")]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_one_rank_row_sharded_solves(dag, gi):
    g = GRAPHS[gi]()
    plan = dag.Plan.from_graph(g, "cuda")
    r, it, ok = RS.pagerank_row_sharded(dag, plan, 0, 1)
    assert ok
    if g.name == "instar":
        k, d = g.n - 1, 0.85
        rstar = np.full(g.n, 1.0 / (g.n + d * k))
        rstar[0] = (1 + d * k) / (g.n + d * k)
    else:
        rstar = oracle.pagerank_fixed_point(g, 0.85, tol=1e-11, threads=4)
        _, it_ref, _, _ = oracle.pagerank(g, oracle.SYNC, tol=1e-6)
        assert abs(it - it_ref) <= 1
    assert float(np.abs(r.double().cpu().numpy() - rstar).sum()) <= 1e-5
    w = I.weights_u32(g, 2)
    src = 1
    dd, it2, ok2 = RS.sssp_row_sharded(dag, plan, src, torch.from_numpy(w.astype(np.uint8)).cuda(), 0, 1)
    _, it2_ref, _, _ = oracle.sssp(g, w, src, oracle.SYNC)
    assert ok2 and it2 == it2_ref
    assert np.array_equal(dd.cpu().numpy().view(np.uint32), oracle.dijkstra(g, w, src))


@pytest.mark.parametrize("world", [2, 3, 8])
def test_ranges_in_turn_equal_the_sync_solve(dag, world):
    # every rank's range computed in turn on one GPU into the same arrays: the new iterate after each
    # sweep is the whole synchronous one, so the solve is the oracle's
    g = I.rmat(14, 16, seed=5)
    plan = dag.Plan.from_graph(g, "cuda")
    ranges = RS.rank_ranges(plan.partition(world))
    assert ranges[0][0] == 0 and ranges[-1][1] == g.n
    r0 = torch.full((g.n,), 1.0 / g.n, device="cuda")
    x = torch.empty_like(r0)
    linked = torch.zeros(1, dtype=torch.float64, device="cuda")
    dag.rank_to_state(plan, r0, x, linked)
    nxt = x.clone()
    lk = float(linked.item())
    sweeps = [RS.gpu_pagerank_sweep(dag, plan, lo, hi) for lo, hi in ranges]
    for it in range(1, 200):
        sums = sum(sw(x, lk, nxt) for sw in sweeps)
        res, lk = (float(v) for v in sums.cpu())
        x, nxt = nxt, x
        if res <= 1e-6:
            break
    r = torch.empty_like(r0)
    dag.state_to_rank(plan, x, r)
    _, it_ref, _, _ = oracle.pagerank(g, oracle.SYNC, tol=1e-6)
    assert abs(it - it_ref) <= 1
    rstar = oracle.pagerank_fixed_point(g, 0.85, tol=1e-11, threads=4)
    assert float(np.abs(r.double().cpu().numpy() - rstar).sum()) <= 1e-5


def test_row_sweep_refuses_a_bad_range(dag):
    g = I.rmat(10, 16, seed=1)
    plan = dag.Plan.from_graph(g, "cuda")
    x = torch.zeros(g.n, device="cuda")
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(dag.DagError):
        dag.pagerank_sweep_rows(plan, 5, 4, x, x.clone(), sums)
    with pytest.raises(dag.DagError):
        dag.pagerank_sweep_rows(plan, 0, g.n + 1, x, x.clone(), sums)
