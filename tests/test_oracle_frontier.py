"""Pins for the frontier Bellman-Ford oracle (CPU only)."""
import os

import numpy as np
import pytest

import oracle
from oracle import frontier
import paper_2110_01409_gb300.inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _row_level_edges(g, changed_prev):
    # edges of rows with at least one in-neighbour changed in the previous sweep (independent count)
    rows = set()
    for v in range(g.n):
        for e in range(g.rowptr[v], g.rowptr[v + 1]):
            if changed_prev[g.colidx[e]]:
                rows.add(v)
                break
    return sum(int(g.rowptr[v + 1] - g.rowptr[v]) for v in rows)


def test_hand_worked_path6():
    g = I.from_edges(6, np.arange(5), np.arange(1, 6), "path6")
    w = np.ones(g.m, dtype=np.uint32)
    with open(os.path.join(GOLDEN, "path6_frontier.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert rows
    for P, TILE, sweeps, edges in rows:
        start = oracle.partition(g, int(P))
        dist, it, ed, ok = frontier.sssp_frontier_sync(g, w, 0, start, int(TILE))
        assert ok and list(dist) == [0, 1, 2, 3, 4, 5]
        # one change per sweep, out-degree 1: always below the dense threshold
        assert list(frontier.sssp_frontier_sync(g, w, 0, start, int(TILE), sparse=None)[2]) == list(ed)
        assert it == int(sweeps) and list(ed) == [int(x) for x in edges.split(",")], (P, TILE, list(ed))


def test_tile_layout_matches_partition_tiles():
    # tiles per block = ceil((rows + edges) / TILE); every edge and row end lands in its own block's tiles
    g = I.rmat(9, 8, seed=4)
    for P, TILE in [(1, 64), (7, 100), (32, 33)]:
        start = oracle.partition(g, P)
        et, rt, nt = frontier.block_tiles(g, start, TILE)
        items = np.diff(start) + np.diff(g.rowptr[start])
        assert np.array_equal(nt, (items + TILE - 1) // TILE)
        base = np.concatenate([[0], np.cumsum(nt)])
        owner = np.searchsorted(start, np.arange(g.n), side="right") - 1
        assert np.all(rt >= base[owner]) and np.all(rt < base[owner + 1])
        src, dst = g.edges()
        assert np.all(et >= base[owner[dst]]) and np.all(et <= rt[dst])


@pytest.mark.parametrize("seed,P,TILE", [(1, 1, 50), (2, 5, 64), (3, 16, 200), (4, 3, 1792)])
def test_frontier_matches_plain_sync_and_dijkstra(seed, P, TILE):
    g = I.rmat(8, 8, seed=seed)
    w = I.weights_u32(g, seed)
    src = int(I.sources(g, 1, seed=seed)[0])
    start = oracle.partition(g, P)
    dist, it, ed, ok = frontier.sssp_frontier_sync(g, w, src, start, TILE, sparse=None)
    assert ok and np.array_equal(dist, oracle.dijkstra(g, w, src))
    d_sync, it_sync, upd, ok2 = oracle.sssp(g, w, src, oracle.SYNC)
    assert ok2 and it == it_sync and np.array_equal(dist, d_sync)
    assert ed[0] == g.m
    # between the row-level frontier and the whole graph, sweep by sweep (plain trajectory replayed)
    n = g.n
    dcur = np.full(n, oracle.INF, dtype=np.int64)
    dcur[src] = 0
    src_e, dst_e = g.edges()
    for s in range(it):
        new = dcur.copy()
        fin = dcur[src_e] != oracle.INF
        np.minimum.at(new, dst_e[fin], np.minimum(dcur[src_e[fin]] + w[fin].astype(np.int64), oracle.INF - 1))
        changed = new < dcur
        if s + 1 < it:
            lo = _row_level_edges(g, changed)
            assert lo <= ed[s + 1] <= g.m, (s, lo, ed[s + 1])
        dcur = new


def test_unreachable_and_single_tile():
    g = I.from_edges(5, [0, 1], [1, 2], "tiny")
    w = np.array([3, 4], dtype=np.uint32)
    start = oracle.partition(g, 1)
    dist, it, ed, ok = frontier.sssp_frontier_sync(g, w, 0, start, 1792)
    assert ok and list(dist) == [0, 3, 7, oracle.INF, oracle.INF] and it == 3
    # one tile: all or nothing; sweep 3 has no tile, since vertex 2 (changed in sweep 2) has no out-edge
    assert list(ed) == [2, 2, 0]


def test_dense_sweeps_run_everything_and_never_undercount():
    # with the dense shortcut a sweep either runs every edge or exactly the marked tiles
    g = I.rmat(10, 16, seed=6)
    w = I.weights_u32(g, 6)
    src = int(I.sources(g, 1, seed=6)[0])
    start = oracle.partition(g, 4)
    d_all, it_all, ed_all, _ = frontier.sssp_frontier_sync(g, w, src, start, 128, sparse=None)
    d_sw, it_sw, ed_sw, ok = frontier.sssp_frontier_sync(g, w, src, start, 128, sparse=4.0)
    assert ok and np.array_equal(d_sw, d_all) and it_sw == it_all
    assert np.all((ed_sw == g.m) | (ed_sw == ed_all))
    assert np.all(ed_sw >= ed_all)
    # with a threshold of 0 every sweep after the first is dense
    ed0 = frontier.sssp_frontier_sync(g, w, src, start, 128, sparse=0.0)[2]
    assert np.all(ed0 == g.m)
