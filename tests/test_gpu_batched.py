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


def test_batched_graph_replays_equal_direct_launches_and_the_oracle(dag, graph):
    # the batched launch is replayed from the plan's CUDA graph of its shape (the default); calls with new
    # buffers, new teleport matrices and a new B replay with their own arguments. In the synchronous form
    # every column's arithmetic is fixed, so replays and direct launches agree bit for bit.
    g = graph
    plan_g = dag.Plan.from_graph(g, "cuda")  # graphs on
    plan_d = dag.Plan.from_graph(g, "cuda")
    plan_d.set_batched_graph(False)
    for B, seed in [(40, 11), (40, 12), (33, 13), (64, 14), (40, 15)]:
        sets = I.ppr_seed_sets(g.n, B, seed=seed)
        V = torch.from_numpy(I.teleport_matrix(g.n, sets)).cuda()
        out = torch.full_like(V, -1.0)  # a fresh output buffer each call
        Rg, itg, stg = dag.ppr_batched(plan_g, V, 0.85, 1e-6, "sync", 0, out=out)
        Rd, itd, std = dag.ppr_batched(plan_d, V.clone(), 0.85, 1e-6, "sync", 0)
        assert stg["graph"] and not std["graph"], (B, stg, std, dag.lib().dag_last_error_message().decode())
        assert stg["converged"] and std["converged"]
        assert torch.equal(Rg, Rd) and torch.equal(itg, itd)
        Vh = V.cpu().numpy().astype(np.float64)
        for c in (0, B - 1):
            rstar = oracle.pagerank_fixed_point(g, 0.85, tele=Vh[:, c])
            assert np.abs(Rg[:, c].cpu().numpy().astype(np.float64) - rstar).sum() <= 1e-5, (B, c)
    # the asynchronous form too (results agree within the parity bound, not bit for bit)
    sets = I.ppr_seed_sets(g.n, 40, seed=16)
    V = torch.from_numpy(I.teleport_matrix(g.n, sets)).cuda()
    Rg, _, stg = dag.ppr_batched(plan_g, V, 0.85, 1e-6, "async", 0)
    assert stg["graph"] and stg["converged"]
    rstar = oracle.pagerank_fixed_point(g, 0.85, tele=V[:, 7].cpu().numpy().astype(np.float64))
    assert np.abs(Rg[:, 7].cpu().numpy().astype(np.float64) - rstar).sum() <= 1e-5
    # Bellman-Ford replays: new sources, new B, both weight widths
    w = I.weights_u32(g, 9)
    for B, seed in [(33, 5), (20, 6)]:
        srcs = torch.from_numpy(I.sources(g, B, seed=seed).view(np.int32)).cuda()
        for wd in (torch.from_numpy(w.view(np.int32)).cuda(), torch.from_numpy(w.astype(np.uint8)).cuda()):
            D, _, st = dag.sssp_batched(plan_g, srcs, wd, "async", 0)
            assert st["graph"] and st["converged"]
            D = D.cpu().numpy().view(np.uint32)
            for c in (0, B - 1):
                assert np.array_equal(D[:, c], oracle.dijkstra(g, w, int(srcs[c])))


@pytest.mark.parametrize("variant,delta", [("sync", 0), ("async", 0), ("delayed", 8)])
def test_sssp_batched_one_byte_weights(dag, graph, variant, delta):
    g = graph
    w = I.weights_u32(g, 9)
    srcs = torch.from_numpy(I.sources(g, 40, seed=8).view(np.int32)).cuda()
    plan = dag.Plan.from_graph(g, "cuda")
    D8, it8, st8 = dag.sssp_batched(plan, srcs, torch.from_numpy(w.astype(np.uint8)).cuda(), variant, delta)
    D4, it4, st4 = dag.sssp_batched(plan, srcs, torch.from_numpy(w.view(np.int32)).cuda(), variant, delta)
    assert st8["converged"] and torch.equal(D8, D4)
    if variant == "sync":
        assert torch.equal(it8, it4)
    D8 = D8.cpu().numpy().view(np.uint32)
    for c in (0, 17, 39):
        assert np.array_equal(D8[:, c], oracle.dijkstra(g, w, int(srcs[c])))


# ---- the wide kernel: 32, 64, 128 or 256 columns, synchronous and asynchronous forms ----
@pytest.mark.parametrize("B", [32, 64, 128, 256])
@pytest.mark.parametrize("variant", ["sync", "async"])
def test_wide_ppr_batched_matches_oracle_and_the_narrow_kernel(dag, graph, B, variant):
    # a warp per share of each tile over all B columns: every checked column within L1 1e-5 of its fp64
    # fixed point; the synchronous form in as many sweeps as the 32-column kernel (within one) and equal
    # values within rounding (a row split between shares adds its partial sums in another order)
    g = graph
    sets = I.ppr_seed_sets(g.n, B, seed=11)
    V = torch.from_numpy(I.teleport_matrix(g.n, sets)).cuda()
    plan = dag.Plan.from_graph(g, "cuda")
    R, iters, st = dag.ppr_batched(plan, V, 0.85, 1e-6, variant, 0)
    assert st["converged"], st
    plan.set_batched_wide(False)
    R2, iters2, st2 = dag.ppr_batched(plan, V, 0.85, 1e-6, variant, 0)
    assert st2["converged"]
    Rn = R.cpu().numpy().astype(np.float64)
    for c in sorted({0, 1, B // 2, B - 1, int(np.argmax(iters.cpu().numpy()))}):
        rstar = oracle.pagerank_fixed_point(g, 0.85, tele=V[:, c].cpu().numpy().astype(np.float64))
        assert np.abs(Rn[:, c] - rstar).sum() <= 1e-5, c
    if variant == "sync":
        # the residual sums differ in their last bits (another summation order), so a column whose
        # residual lands at the tolerance may take one sweep more in one kernel than in the other
        assert int(np.abs(iters.cpu().numpy() - iters2.cpu().numpy()).max()) <= 1
        assert float((R - R2).abs().max()) <= 1e-5
    assert st["column_sweeps"] == int(iters.sum())


@pytest.mark.parametrize("B", [32, 64, 256])
@pytest.mark.parametrize("variant", ["sync", "async"])
@pytest.mark.parametrize("u8", [True, False])
def test_wide_sssp_batched_bit_exact(dag, B, variant, u8):
    # hub rows longer than a tile and tiles inside one row: RMAT scale 14 with its heavy in-degree head
    g = I.rmat(14, 16, seed=8)
    w = I.weights_u32(g, 12)
    srcs = I.sources(g, B, seed=13)
    plan = dag.Plan.from_graph(g, "cuda")
    wd = torch.from_numpy(w.astype(np.uint8) if u8 else w.view(np.int32)).cuda()
    D, iters, st = dag.sssp_batched(plan, torch.from_numpy(srcs.view(np.int32)).cuda(), wd, variant, 0)
    assert st["converged"]
    D = D.cpu().numpy().view(np.uint32)
    its = iters.cpu().numpy()
    for c in sorted({0, 1, B // 3, B - 1}):
        assert np.array_equal(D[:, c], oracle.dijkstra(g, w, int(srcs[c]))), c
        if variant == "sync":
            _, it, _, _ = oracle.sssp(g, w, int(srcs[c]), oracle.SYNC)
            assert its[c] == it
    plan.set_batched_wide(False)
    D2, _, _ = dag.sssp_batched(plan, torch.from_numpy(srcs.view(np.int32)).cuda(), wd, variant, 0)
    assert np.array_equal(D, D2.cpu().numpy().view(np.uint32))


def test_wide_batched_tiny_graphs(dag):
    # rows of no in-edges, a graph smaller than one tile, and the delayed form on the 32-column kernel
    g = I.from_edges(6, [0, 1, 2, 0], [1, 2, 3, 3], "tiny")
    plan = dag.Plan.from_graph(g, "cuda")
    V = np.zeros((6, 32), dtype=np.float32)
    V[np.arange(32) % 6, np.arange(32)] = 1.0
    for variant, delta in (("sync", 0), ("async", 0), ("delayed", 4)):
        # (tol 1e-6: with ranks near 0.2 the FP32 residual of six rows cannot fall much below 1e-7)
        R, _, st = dag.ppr_batched(plan, torch.from_numpy(V).cuda(), 0.85, 1e-6, variant, delta)
        assert st["converged"]
        R = R.cpu().numpy()
        for c in (0, 1, 5, 31):
            rstar = oracle.pagerank_fixed_point(g, 0.85, tele=V[:, c].astype(np.float64))
            assert np.abs(R[:, c] - rstar).sum() <= 1e-5, (variant, c)
