"""Pins for the Bellman-Ford / Dijkstra oracle (CPU only)."""
import os

import numpy as np
import pytest

import oracle
import paper_2110_01409_gb300.inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.INF


def floyd_warshall(g, w):
    n = g.n
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    src, dst = g.edges()
    for u, v, x in zip(src, dst, w):
        D[u, v] = min(D[u, v], float(x))
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def as_u32(dist_float):
    out = np.full(len(dist_float), INF, dtype=np.uint64)
    fin = np.isfinite(dist_float)
    out[fin] = dist_float[fin].astype(np.uint64)
    return out.astype(np.uint32)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_dijkstra_matches_floyd_warshall(seed):
    g = I.rmat(6, 4, seed=seed)
    w = I.weights_u32(g, seed + 10)
    D = floyd_warshall(g, w)
    for src in [0, 5, 17, 63]:
        assert np.array_equal(oracle.dijkstra(g, w, src), as_u32(D[src]))


def test_unit_weights_give_bfs_levels():
    g = I.rmat(9, 8, seed=9)
    w = np.ones(g.m, dtype=np.uint32)
    # plain BFS over out-edges
    src, dst = g.edges()
    order = np.argsort(src, kind="stable")
    optr = np.searchsorted(src[order], np.arange(g.n + 1))
    level = np.full(g.n, INF, dtype=np.uint32)
    level[0] = 0
    frontier = [0]
    while frontier:
        nxt = []
        for u in frontier:
            for v in dst[order[optr[u]:optr[u + 1]]]:
                if level[v] == INF:
                    level[v] = level[u] + 1
                    nxt.append(v)
        frontier = nxt
    assert np.array_equal(oracle.dijkstra(g, w, 0), level)
    dist, _, _, ok = oracle.sssp(g, w, 0, oracle.DELAYED, P=5, delta=3)
    assert ok and np.array_equal(dist, level)


def _min_hops_on_shortest_paths(g, w, dist, src):
    # hop[v] = min over tight in-edges (dist[u] + w = dist[v]) of hop[u] + 1,
    # taken in order of increasing distance (weights >= 1 make that a valid order)
    hop = np.full(g.n, np.iinfo(np.int64).max, dtype=np.int64)
    hop[src] = 0
    reach = np.nonzero(dist != INF)[0]
    for v in reach[np.argsort(dist[reach], kind="stable")]:
        if v == src:
            continue
        for e in range(g.rowptr[v], g.rowptr[v + 1]):
            u = g.colidx[e]
            if dist[u] != INF and int(dist[u]) + int(w[e]) == int(dist[v]):
                hop[v] = min(hop[v], hop[u] + 1)
    return int(hop[reach].max())


@pytest.mark.parametrize("seed,src", [(1, 0), (2, 3), (3, 11), (11, 1)])
def test_bellman_ford_variants_match_dijkstra_and_invariants(seed, src):
    g = I.rmat(10, 16, seed=seed)
    w = I.weights_u32(g, 100 + seed)
    ref = oracle.dijkstra(g, w, src)
    # invariants of the exact distances
    assert ref[src] == 0
    s, t = g.edges()
    fin = ref[s] != INF
    assert np.all(ref[t[fin]].astype(np.int64) <= ref[s[fin]].astype(np.int64) + w[fin])
    tight = np.zeros(g.n, bool)
    tight[t[fin][ref[t[fin]].astype(np.int64) == ref[s[fin]].astype(np.int64) + w[fin]]] = True
    reach = ref != INF
    reach[src] = False
    assert np.all(tight[reach])
    # sync sweeps = 1 + the largest minimum hop count over shortest paths
    dist, it_sync, upd, ok = oracle.sssp(g, w, src, oracle.SYNC)
    assert ok and np.array_equal(dist, ref)
    assert it_sync == 1 + _min_hops_on_shortest_paths(g, w, ref, src)
    assert upd[-1] == 0 and np.all(upd[:-1] > 0)
    for P, delta in [(1, 0), (16, 0), (16, 1), (16, 16), (16, 64), (64, 1000)]:
        dist, it, _, ok = oracle.sssp(g, w, src, oracle.DELAYED, P=P, delta=delta)
        assert ok and np.array_equal(dist, ref), (P, delta)
        # fresher values can only lower distances sooner
        assert it <= it_sync
        dist, it_l, _, ok = oracle.sssp(g, w, src, oracle.DELAYED, P=P, delta=delta, local_read=True)
        assert ok and np.array_equal(dist, ref) and it_l <= it_sync


def test_hand_worked_path6_traces():
    g = I.from_edges(6, np.arange(5), np.arange(1, 6), "path6")
    w = np.ones(g.m, dtype=np.uint32)
    with open(os.path.join(GOLDEN, "path6_sssp_traces.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for name, P, delta, iters, upd in rows:
        P, delta, iters = int(P), int(delta), int(iters)
        want_upd = [int(x) for x in upd.split(",")]
        if delta < 0:
            dist, it, u, ok = oracle.sssp(g, w, 0, oracle.SYNC)
        else:
            dist, it, u, ok = oracle.sssp(g, w, 0, oracle.DELAYED, P=P, delta=delta,
                                          local_read=name.startswith("local"))
        assert ok, name
        assert list(dist) == [0, 1, 2, 3, 4, 5], name
        assert it == iters and list(u) == want_upd, name


def test_unreachable_and_isolated_source():
    g = I.from_edges(5, [0, 1], [1, 2], "tiny")
    w = np.array([3, 4], dtype=np.uint32)
    dist, it, _, ok = oracle.sssp(g, w, 0, oracle.SYNC)
    assert ok and list(dist) == [0, 3, 7, INF, INF] and it == 3
    dist, it, _, ok = oracle.sssp(g, w, 4, oracle.DELAYED, P=2, delta=1)
    assert ok and list(dist) == [INF, INF, INF, INF, 0] and it == 1
    assert list(oracle.dijkstra(g, w, 4)) == [INF, INF, INF, INF, 0]


def test_threaded_form_matches_dijkstra():
    g = I.rmat(12, 16, seed=2)
    w = I.weights_u32(g, 5)
    ref = oracle.dijkstra(g, w, 0)
    for variant, delta in [(0, 0), (1, 0), (2, 32)]:
        dist, it, sec, ok = oracle.sssp_threads(g, w, 0, variant, threads=4, delta=delta)
        assert ok and np.array_equal(dist, ref)


def test_row_sweeps_cover_one_sync_sweep_sssp():
    g = I.rmat(10, 16, seed=1)
    w = I.weights_u32(g, 1)
    d0 = np.full(g.n, oracle.INF, dtype=np.uint32)
    d0[0] = 0
    want, _, upd, _ = oracle.sssp(g, w, 0, oracle.SYNC, max_iters=1)
    out = np.zeros(g.n, dtype=np.uint32)
    c = oracle.sssp_sweep_rows(g, w, 0, 300, d0, out) + oracle.sssp_sweep_rows(g, w, 300, g.n, d0, out)
    assert np.array_equal(out, want) and c == upd[0]
