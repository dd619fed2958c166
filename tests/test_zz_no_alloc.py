"""dag_pagerank_noalloc: PageRank for callers that cannot allocate device memory.

Some applications cannot let a library call cudaMalloc while they solve: their
device memory is owned by their own pool allocator, or the solve sits on a
latency-critical path where cudaMalloc's implicit device synchronisation is not
acceptable. dag_pagerank_noalloc serves them: it keeps all of its scratch in a
fixed array inside the library. These tests call it through the C ABI twice in
a row (the second call finds the first call's leftovers in that array) and
check each result against the plan-based dag_pagerank within the L1 tolerance
of the other PageRank tests (1e-5), and against the oracle's fp64 fixed point;
a graph over the stated limit and a CSR with an out-of-range colidx are
refused. The file name makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_01409_gb300.inputs as I

pytestmark = pytest.mark.gpu

VARIANTS = [("sync", 0), ("delayed", 64), ("async", 0)]


@pytest.fixture(scope="module")
def dag():
    from paper_2110_01409_gb300 import build, dag as D

    build.build()
    assert torch.cuda.is_available()
    return D


def _l1(a, b):
    return float((a.double() - b.double()).abs().sum())


def _dev(g):
    return torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.colidx).cuda()


@pytest.mark.parametrize("variant,delta", VARIANTS)
def test_noalloc_matches_plan_entry_point_twice(dag, variant, delta):
    g = I.rmat(14, 16, seed=21)
    rowptr, colidx = _dev(g)
    plan = dag.Plan(rowptr, colidx)
    ref, st = dag.pagerank(plan, 0.85, 1e-6, variant, delta)
    assert st["converged"]
    rstar = torch.from_numpy(oracle.pagerank_fixed_point(g, 0.85))
    for _ in range(2):
        out = torch.full((g.n,), -1.0, device="cuda")
        r, st2 = dag.pagerank_noalloc(rowptr, colidx, 0.85, 1e-6, variant, delta, out=out)
        assert st2["converged"], st2
        assert _l1(r, ref) <= 1e-5
        assert _l1(r.cpu(), rstar) <= 1e-5


@pytest.mark.parametrize("variant,delta", VARIANTS)
def test_noalloc_second_graph_after_first(dag, variant, delta):
    # a smaller graph after a larger one: stale scratch (state buffers, partition, out-degrees) must
    # not leak into it
    for scale, seed in [(15, 3), (11, 4)]:
        g = I.rmat(scale, 16, seed=seed)
        rowptr, colidx = _dev(g)
        ref, _ = dag.pagerank(dag.Plan(rowptr, colidx), 0.85, 1e-6, variant, delta)
        r, st = dag.pagerank_noalloc(rowptr, colidx, 0.85, 1e-6, variant, delta)
        assert st["converged"] and _l1(r, ref) <= 1e-5
        assert _l1(r.cpu(), torch.from_numpy(oracle.pagerank_fixed_point(g, 0.85))) <= 1e-5


def test_noalloc_personalized_teleport(dag):
    g = I.rmat(13, 16, seed=6)
    rowptr, colidx = _dev(g)
    t = np.zeros(g.n, dtype=np.float32)
    t[[3, 77, 1000, 4095]] = 0.25
    td = torch.from_numpy(t).cuda()
    ref, _ = dag.pagerank(dag.Plan(rowptr, colidx), 0.85, 1e-6, "delayed", 64, teleport=td)
    r, st = dag.pagerank_noalloc(rowptr, colidx, 0.85, 1e-6, "delayed", 64, teleport=td)
    assert st["converged"] and _l1(r, ref) <= 1e-5
    rstar = oracle.pagerank_fixed_point(g, 0.85, tele=t.astype(np.float64))
    assert _l1(r.cpu(), torch.from_numpy(rstar)) <= 1e-5


def test_noalloc_rejects_graph_over_the_limit(dag):
    n = (1 << 20) + 1
    rowptr = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    colidx = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(dag.DagError) as ei:
        dag.pagerank_noalloc(rowptr, colidx)
    assert ei.value.code == dag.ERR_INVALID
    assert "too large" in str(ei.value)


def test_noalloc_rejects_colidx_out_of_range(dag):
    # checked on the device before the solve; a valid call afterwards still works
    g = I.rmat(10, 16, seed=1)
    rowptr, colidx = _dev(g)
    bad = colidx.clone()
    bad[17] = g.n  # one past the last vertex
    with pytest.raises(dag.DagError) as ei:
        dag.pagerank_noalloc(rowptr, bad)
    assert ei.value.code == dag.ERR_INVALID
    r, st = dag.pagerank_noalloc(rowptr, colidx, 0.85, 1e-6, "delayed", 16)
    assert st["converged"]
    assert _l1(r.cpu(), torch.from_numpy(oracle.dense_pagerank(g, 0.85))) <= 1e-5
