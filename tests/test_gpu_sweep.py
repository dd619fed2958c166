"""GPU parity of the single-vector sweeps against the CPU oracle (through the C ABI).

PageRank: L1 distance to the fp64 fixed point <= 1e-5 at tol 1e-6 (FP32 ranks;
the bound follows from the Jacobi contraction, tol*d/(1-d) = 5.7e-6, plus FP32
rounding of O(1e-7)). Bellman-Ford: bit-exact against Dijkstra. Sync sweep
counts: equal to the oracle's for SSSP (deterministic), within one for
PageRank (FP32 vs fp64 residual at the threshold).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_01409_gb300.inputs as I

pytestmark = pytest.mark.gpu

VARIANTS_PR = [("sync", 0), ("async", 0), ("delayed", 1), ("delayed", 16), ("delayed", 64), ("delayed", 1000),
               ("delayed", 100000), ("delayed", 37)]


@pytest.fixture(scope="module")
def dag():
    from paper_2110_01409_gb300 import build, dag as D

    build.build()
    assert torch.cuda.is_available()
    return D


def _plan(dag, g, **kw):
    return dag.Plan.from_graph(g, "cuda", **kw)


def _l1(r_gpu, ref):
    return float(np.abs(r_gpu.detach().cpu().numpy().astype(np.float64) - ref).sum())


def _w_dev(w):
    return torch.from_numpy(np.ascontiguousarray(w).view(np.int32)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("variant,delta", VARIANTS_PR)
def test_pagerank_scale10_config(dag, variant, delta):
    g = I.rmat(10, 16, seed=1)
    plan = _plan(dag, g)
    rstar = oracle.dense_pagerank(g, 0.85)
    r, st = dag.pagerank(plan, 0.85, 1e-6, variant, delta)
    assert st["converged"], st
    assert _l1(r, rstar) <= 1e-5
    assert abs(float(r.double().sum()) - 1.0) <= 1e-5
    if variant == "sync":
        _, it, _, _ = oracle.pagerank(g, oracle.SYNC, tol=1e-6)
        assert abs(st["iters"] - it) <= 1


@pytest.mark.parametrize("maker", [
    lambda: I.rmat(14, 16, seed=7),
    lambda: I.rmat(13, 4, seed=8),
    lambda: I.erdos_renyi(20000, 16, seed=3),
    lambda: I.banded(30011, 15, 1024, 1, seed=3),
])
@pytest.mark.parametrize("variant,delta", [("sync", 0), ("async", 0), ("delayed", 32), ("delayed", 4096)])
def test_pagerank_many_tiles_ragged(dag, maker, variant, delta):
    g = maker()
    plan = _plan(dag, g)
    rstar = oracle.pagerank_fixed_point(g, 0.85)
    r, st = dag.pagerank(plan, 0.85, 1e-6, variant, delta)
    assert st["converged"]
    assert _l1(r, rstar) <= 1e-5, (st, _l1(r, rstar))


def _from_edges(n, s, t):
    return I.from_edges(n, np.asarray(s), np.asarray(t))


@pytest.mark.parametrize("variant,delta", VARIANTS_PR)
def test_pagerank_closed_forms(dag, variant, delta):
    n = 5000
    cyc = _from_edges(n, np.arange(n), (np.arange(n) + 1) % n)
    r, st = dag.pagerank(_plan(dag, cyc), 0.85, 1e-7, variant, delta)
    assert np.max(np.abs(r.cpu().numpy() - 1.0 / n)) <= 1e-9
    k = 9000  # in-star: hub row of 9000 in-edges spans several tiles
    star = _from_edges(k + 1, np.arange(1, k + 1), np.zeros(k, int))
    r, st = dag.pagerank(_plan(dag, star), 0.85, 1e-7, variant, delta)
    want = np.full(k + 1, 1.0 / (k + 1 + 0.85 * k))
    want[0] = (1 + 0.85 * k) / (k + 1 + 0.85 * k)
    assert np.max(np.abs(r.cpu().numpy() - want)) <= 1e-6 * want.max()
    # personalized: e_s on a cycle
    n2, s = 64, 5
    cyc2 = _from_edges(n2, np.arange(n2), (np.arange(n2) + 1) % n2)
    tele = torch.zeros(n2, device="cuda")
    tele[s] = 1.0
    r, _ = dag.pagerank(_plan(dag, cyc2), 0.85, 1e-8, variant, delta, teleport=tele)
    want = np.array([(1 - 0.85) * 0.85 ** ((v - s) % n2) / (1 - 0.85 ** n2) for v in range(n2)])
    assert np.max(np.abs(r.cpu().numpy() - want)) <= 1e-6


def test_pagerank_weighted_and_personalized(dag):
    g = I.rmat(12, 16, seed=11)
    w = I.weights_f32(g, 5)
    val, s = oracle.normalize(g, w.astype(np.float64))
    tele = np.zeros(g.n)
    tele[[3, 77, 1000]] = 1.0 / 3
    rstar = oracle.pagerank_fixed_point(g, 0.85, tele, val)
    plan = _plan(dag, g)
    for variant, delta in [("sync", 0), ("async", 0), ("delayed", 64)]:
        r, st = dag.pagerank(plan, 0.85, 1e-6, variant, delta, teleport=torch.tensor(tele, dtype=torch.float32,
                             device="cuda"), val=torch.tensor(val, dtype=torch.float32, device="cuda"))
        assert st["converged"] and _l1(r, rstar) <= 1e-5


@pytest.mark.parametrize("variant,delta", [("sync", 0), ("async", 0), ("delayed", 1), ("delayed", 16),
                                           ("delayed", 64), ("delayed", 5000), ("delayed", 33)])
def test_sssp_bit_exact(dag, variant, delta):
    for g, src in [(I.rmat(10, 16, seed=1), 0), (I.rmat(14, 16, seed=2), 5), (I.banded(20000, 15, 1024, 1, 3), 7)]:
        w = I.weights_u32(g, 1)
        plan = _plan(dag, g)
        ref = oracle.dijkstra(g, w, src)
        d, st = dag.sssp(plan, src, _w_dev(w), variant, delta)
        assert st["converged"]
        assert np.array_equal(_u32(d), ref)
        if variant == "sync":
            _, it, _, _ = oracle.sssp(g, w, src, oracle.SYNC)
            assert st["iters"] == it
        else:
            _, it_sync, _, _ = oracle.sssp(g, w, src, oracle.SYNC)
            assert st["iters"] <= it_sync


def test_edge_cases(dag):
    # one vertex, no edges
    g1 = _from_edges(1, [], [])
    r, st = dag.pagerank(_plan(dag, g1), 0.85, 1e-6, "delayed", 16)
    assert st["converged"] and abs(float(r[0]) - 1.0) < 1e-6
    d, st = dag.sssp(_plan(dag, g1), 0, None, "async", 0)
    assert int(_u32(d)[0]) == 0
    # no edges at all: every vertex dangling, r = 1/n
    g0 = _from_edges(1000, [], [])
    r, st = dag.pagerank(_plan(dag, g0), 0.85, 1e-6, "delayed", 64)
    assert np.max(np.abs(r.cpu().numpy() - 1e-3)) < 1e-9
    # isolated source: everything else unreachable
    g = _from_edges(6, [0, 1, 2], [1, 2, 3])
    w = np.array([5, 6, 7], dtype=np.uint32)
    d, st = dag.sssp(_plan(dag, g), 4, _w_dev(w), "delayed", 1)
    assert list(_u32(d)) == [0xFFFFFFFF] * 4 + [0, 0xFFFFFFFF] and st["iters"] == 1
    d, st = dag.sssp(_plan(dag, g), 0, _w_dev(w), "sync", 0)
    assert list(_u32(d)) == [0, 5, 11, 18, 0xFFFFFFFF, 0xFFFFFFFF] and st["iters"] == 4


def test_partition_and_out_degree_match_oracle(dag):
    g = I.rmat(14, 16, seed=3)
    plan = _plan(dag, g)
    for P in [1, 7, 152, 1216, 5000]:
        assert np.array_equal(plan.partition(P), oracle.partition(g, P))
    assert np.array_equal(plan.out_degree().cpu().numpy(), oracle.out_degree(g))


def test_not_converged_returns_last_iterate(dag):
    g = I.rmat(12, 16, seed=4)
    plan = _plan(dag, g)
    r, st = dag.pagerank(plan, 0.85, 1e-6, "sync", 0, max_iters=2)
    assert not st["converged"] and st["err"] == dag.ERR_NOT_CONVERGED and st["iters"] == 2
    r2, _, _, _ = oracle.pagerank(g, oracle.SYNC, tol=0.0, max_iters=2)
    assert _l1(r, r2) <= 1e-5
    # warm start from that iterate finishes the job
    r, st = dag.pagerank(plan, 0.85, 1e-6, "sync", 0, out=r, warm_start=True)
    assert st["converged"] and _l1(r, oracle.pagerank_fixed_point(g)) <= 1e-5


def test_invalid_arguments_rejected(dag):
    g = I.rmat(8, 4, seed=1)
    plan = _plan(dag, g)
    with pytest.raises(dag.DagError):
        dag.pagerank(plan, 1.5, 1e-6, "sync", 0)
    with pytest.raises(dag.DagError):
        dag.pagerank(plan, 0.85, 1e-6, "delayed", -1)
    with pytest.raises(dag.DagError):
        dag.sssp(plan, g.n + 3, _w_dev(I.weights_u32(g, 1)))
    bad = torch.from_numpy(g.colidx.copy()).cuda()
    bad[5] = g.n + 10
    with pytest.raises(dag.DagError):
        dag.Plan(torch.from_numpy(g.rowptr).cuda(), bad)


def test_barrier_timeout_is_reported_and_context_survives(dag):
    g = I.rmat(10, 16, seed=1)
    plan = _plan(dag, g)
    plan.debug_skip_barrier_once(100)
    with pytest.raises(dag.DagError) as ei:
        dag.pagerank(plan, 0.85, 1e-6, "delayed", 16)
    assert ei.value.code == dag.ERR_BARRIER_TIMEOUT
    r, st = dag.pagerank(plan, 0.85, 1e-6, "delayed", 16)
    assert st["converged"] and _l1(r, oracle.dense_pagerank(g)) <= 1e-5


@pytest.mark.parametrize("algo", ["pagerank", "sssp8"])
def test_staging_wait_timeout_is_reported_and_context_survives(dag, algo):
    # the asynchronous sweep's bounded wait for a tile's TMA copies runs out (its mbarrier phase is
    # announced 16 bytes short); the call reports it and the next solve on the plan is fine
    g = I.rmat(12, 16, seed=2)
    plan = _plan(dag, g)
    w8 = torch.from_numpy(I.weights_u32(g, 1).astype(np.uint8)).cuda()

    def solve():
        if algo == "pagerank":
            return dag.pagerank(plan, 0.85, 1e-6, "async", 0)
        return dag.sssp(plan, 3, w8, "async", 0)

    plan.debug_stall_staging_once(100)
    with pytest.raises(dag.DagError) as ei:
        solve()
    assert ei.value.code == dag.ERR_BARRIER_TIMEOUT
    out, st = solve()
    assert st["converged"]
    if algo == "pagerank":
        assert _l1(out, oracle.pagerank_fixed_point(g, 0.85)) <= 1e-5
    else:
        assert np.array_equal(_u32(out), oracle.dijkstra(g, I.weights_u32(g, 1), 3))


def test_flush_counts_follow_delta(dag):
    g = I.rmat(18, 16, seed=5)  # several tiles per CTA
    plan = _plan(dag, g)
    P = plan.workers("delayed", 10 ** 7)
    _, st = dag.pagerank(plan, 0.85, 1e-6, "delayed", 10 ** 7)
    # delta >= rows per CTA: one flush per non-empty block per sweep (Sec. III-B's "synchronous" end)
    start = plan.partition(P)
    nonempty = int(np.sum(np.diff(start) > 0))
    assert st["flushes"] == nonempty * st["iters"]
    # delta below a tile's rows: tiles complete at most delta rows and a flush follows as soon as the
    # buffer holds >= delta, so each flush carries delta .. 2 delta - 1 rows (fewer only at a block end):
    # n / (2 delta - 1) <= flushes per sweep <= n / delta + blocks
    for delta in (16, 64):
        _, st_d = dag.pagerank(plan, 0.85, 1e-6, "delayed", delta)
        assert st_d["converged"]
        per_sweep = st_d["flushes"] / st_d["iters"]
        assert g.n / (2 * delta - 1) <= per_sweep <= g.n / delta + st_d["workers"], (delta, per_sweep)


@pytest.mark.parametrize("variant,delta", [("sync", 0), ("async", 0), ("delayed", 16), ("delayed", 5000)])
def test_sssp_u8_weights_bit_exact(dag, variant, delta):
    # dag_sssp_u8 reads one byte per edge; results equal Dijkstra on the same weights
    for g, src in [(I.rmat(14, 16, seed=2), 5), (I.erdos_renyi(30000, 16, seed=3), 11)]:
        w = I.weights_u32(g, 1)
        plan = _plan(dag, g)
        ref = oracle.dijkstra(g, w, src)
        d, st = dag.sssp(plan, src, torch.from_numpy(w.astype(np.uint8)).cuda(), variant, delta)
        assert st["converged"] and np.array_equal(_u32(d), ref)
        if variant == "sync":
            _, it, _, _ = oracle.sssp(g, w, src, oracle.SYNC)
            assert st["iters"] == it


def test_gather_probe_runs(dag):
    g = I.rmat(14, 16, seed=2)
    plan = _plan(dag, g)
    x = torch.ones(g.n, device="cuda")
    for coherent in (True, False):
        ms = dag.probe_gather(plan, x, coherent=coherent, repeats=2)
        assert 0.0 < ms < 1000.0


@pytest.mark.parametrize("delta", [64, 4096, 10 ** 6])
def test_local_reads_parity(dag, delta):
    # Sec. III-C local reads: a CTA reads its own unflushed values from its buffer
    for g in [I.rmat(14, 16, seed=7), I.banded(30011, 15, 1024, 1, seed=3)]:
        plan = _plan(dag, g)
        rstar = oracle.pagerank_fixed_point(g, 0.85)
        r, st = dag.pagerank(plan, 0.85, 1e-6, "delayed", delta, reads="local")
        assert st["converged"] and _l1(r, rstar) <= 1e-5
        w = I.weights_u32(g, 1)
        ref = oracle.dijkstra(g, w, 5)
        d, st2 = dag.sssp(plan, 5, _w_dev(w), "delayed", delta, reads="local")
        assert st2["converged"] and np.array_equal(_u32(d), ref)
        _, it_sync, _, _ = oracle.sssp(g, w, 5, oracle.SYNC)
        assert st2["iters"] <= it_sync


@pytest.mark.parametrize("reads", ["own_l1", "cached"])
@pytest.mark.parametrize("algo", ["pagerank", "sssp", "sssp8"])
def test_async_own_block_l1_parity(dag, algo, reads):
    # async form (CTA tiles) with the CTA's own block read through L1 (own_l1), or every gather an ordinary
    # load refreshed by the grid barrier (cached): same fixed point / exact distances, and no more
    # Bellman-Ford sweeps than the synchronous form (every value read is at most one sweep old)
    for g in [I.rmat(14, 16, seed=8), I.banded(30011, 15, 1024, 1, seed=4), I.banded(1 << 17, 15, 16, 1, seed=4)]:
        plan = _plan(dag, g)
        if algo == "pagerank":
            r, st = dag.pagerank(plan, 0.85, 1e-6, "async", 0, reads=reads)
            assert st["converged"] and _l1(r, oracle.pagerank_fixed_point(g, 0.85)) <= 1e-5
            continue
        w = I.weights_u32(g, 2)
        ref = oracle.dijkstra(g, w, 3)
        wd = torch.from_numpy(w.astype(np.uint8)).cuda() if algo == "sssp8" else _w_dev(w)
        d, st = dag.sssp(plan, 3, wd, "async", 0, reads=reads)
        assert st["converged"] and np.array_equal(_u32(d), ref)
        _, it_sync, _, _ = oracle.sssp(g, w, 3, oracle.SYNC)
        assert st["iters"] <= it_sync


@pytest.mark.parametrize("P", [1, 32, 152, 700])
def test_access_matrix_counts_exact(dag, P):
    # Fig. 5: reads by block i (owner of v) of block j's vertices (owner of u), for edges u -> v
    for g in [I.rmat(13, 16, seed=3), I.banded(20011, 15, 1024, 1, seed=3)]:
        plan = _plan(dag, g)
        got = dag.access_matrix(plan, P).cpu().numpy()
        start = oracle.partition(g, P)
        src, dst = g.edges()
        own = lambda x: np.searchsorted(start, x, side="right") - 1  # noqa: E731
        want = np.bincount(own(dst) * P + own(src), minlength=P * P).reshape(P, P)
        assert np.array_equal(got, want)
        assert got.sum() == g.m


def test_access_matrix_locality_rmat_vs_banded(dag):
    # Sec. IV-C: a clustered graph's reads stay mostly on the diagonal, an RMAT graph's do not
    rm = dag.locality(dag.access_matrix(_plan(dag, I.rmat(16, 16, seed=5)), 32))
    bd = dag.locality(dag.access_matrix(_plan(dag, I.banded(1 << 16, 15, 1024, 1, seed=5)), 32))
    assert bd["diag_share"] > 0.6 and bd["marked_rows"] == 32
    assert rm["diag_share"] < 0.1


def test_autotune_cache_and_locality_cutoff(dag, tmp_path):
    from paper_2110_01409_gb300 import autotune

    cache = str(tmp_path / "tune.json")
    plan = _plan(dag, I.banded(1 << 16, 15, 16, 1, seed=6))  # band 16: local even at thousands of blocks
    c1 = autotune.tune(plan, "pagerank", worker_fractions=[1.0], trials=1, cache=cache, tol=1e-6)
    want = {autotune._norm(c) for c in autotune.SINGLE_CANDIDATES}
    assert {(r["variant"], r["delta"], r["reads"], r["warp_tile"]) for r in c1["candidates"]} == want
    assert (c1["variant"], c1["delta"], c1["reads"], c1["warp_tile"]) in want
    c2 = autotune.tune(plan, "pagerank", worker_fractions=[1.0], trials=1, cache=cache, tol=1e-6)
    assert c2 == c1  # served from the cache
    c3 = autotune.tune(plan, "pagerank", worker_fractions=[1.0], trials=1, cache=None, tol=1e-6,
                       locality_cutoff=0.5)
    assert c3["locality"]["diag_share"] > 0.5
    assert all(r["variant"] != "delayed" for r in c3["candidates"])


def test_last_status_copied_on_the_device(dag):
    # dag_plan_last_status: the last solve's (err, converged, sweeps) into a device array, no host wait
    g = I.rmat(12, 16, seed=4)
    plan = _plan(dag, g)
    st_dev = torch.full((2, 3), -7, dtype=torch.int32, device="cuda")
    _, st = dag.pagerank(plan, 0.85, 1e-6, "async", 0)
    dag.pagerank(plan, 0.85, 1e-6, "async", 0, stats=False)
    plan.last_status_to(st_dev[0])
    dag.pagerank(plan, 0.85, 1e-6, "sync", 0, max_iters=2, stats=False)  # stops before the rule is met
    plan.last_status_to(st_dev[1])
    got = st_dev.cpu().numpy()
    assert got[0, 0] == 0 and got[0, 1] == 1 and got[0, 2] > 2
    assert got[1, 0] == 0 and got[1, 1] == 0 and got[1, 2] == 2
