"""Frontier (conditionally processed) Bellman-Ford: the synchronous sweep with
work skipped where no input changed (Sec. V names conditionally written
updates as the next pull-style case for the method).

TEST INFRASTRUCTURE (see the package docstring). Plain Python/numpy, fp-free.

Reading (the paper gives no algorithm for it). Work is grouped as the GPU
groups it: the static partition of Sec. III-A (block p owns rows
[start[p], start[p+1])), and inside a block the merge-path order of its
items, where row v contributes its in-edges (rowptr[v] .. rowptr[v+1]-1) and
then one row-end item; tile k of block p is the block's items
[k*TILE, (k+1)*TILE), and tiles are numbered globally block after block.
Sweep 0 processes every tile. Sweep s >= 1 processes a tile when it holds an
in-edge u -> v whose source u got a smaller distance in sweep s-1, or lies
between such an edge's tile and the tile holding v's row end. A processed tile
relaxes its edges (a row whose start lies in a skipped tile takes only the
edges of processed tiles); a skipped tile leaves its rows as they are.
Dense sweeps: when the out-degrees of the rows changed in sweep s-1 sum to
more than `sparse` per tile, sweep s processes every tile (such changes reach
nearly every tile anyway, and marking them would cost more than it saves);
`sparse=None` never takes that shortcut.

For the synchronous sweep this gives exactly the plain trajectory: a row none
of whose in-neighbours changed cannot change, and edges from unchanged
sources cannot lower a row below its current value. What it changes is how
many edges each sweep touches, which this module counts exactly.
"""
from __future__ import annotations

import numpy as np

INF = 0xFFFFFFFF


def block_tiles(g, start, TILE):
    """Tile layout of the partition: for every in-edge its tile, for every row
    the tile of its row-end item, and the number of tiles per block."""
    n, rowptr = g.n, g.rowptr
    P = len(start) - 1
    edge_tile = np.empty(g.m, dtype=np.int64)
    end_tile = np.empty(n, dtype=np.int64)
    ntiles = np.zeros(P, dtype=np.int64)
    base = 0
    for p in range(P):
        r0, r1 = int(start[p]), int(start[p + 1])
        e0 = int(rowptr[r0])
        items = (int(rowptr[r1]) - e0) + (r1 - r0)
        ntiles[p] = (items + TILE - 1) // TILE
        for v in range(r0, r1):
            before = v - r0  # row-end items of the block's earlier rows
            for e in range(int(rowptr[v]), int(rowptr[v + 1])):
                edge_tile[e] = base + ((e - e0) + before) // TILE
            end_tile[v] = base + ((int(rowptr[v + 1]) - e0) + before) // TILE
        base += int(ntiles[p])
    return edge_tile, end_tile, ntiles


def sssp_frontier_sync(g, w, src, start, TILE, max_iters=None, sparse=4.0):
    """Synchronous frontier Bellman-Ford. Returns (dist uint32, sweeps, edges
    processed per sweep, converged). Distances saturate at INF - 1 as in the
    plain oracle; INF marks unreachable vertices."""
    n, m = g.n, g.m
    rowptr, colidx = g.rowptr, g.colidx
    w = np.asarray(w, dtype=np.int64)
    edge_tile, end_tile, ntiles = block_tiles(g, start, TILE)
    T = int(ntiles.sum())
    edges_in_tile = np.bincount(edge_tile, minlength=T) if m else np.zeros(T, dtype=np.int64)
    row_of_edge = np.repeat(np.arange(n), np.diff(rowptr))
    max_iters = n + 1 if max_iters is None else max_iters
    dist = np.full(n, INF, dtype=np.int64)
    dist[src] = 0
    active = np.ones(T, dtype=bool)
    edges, it, ok = [], 0, False
    src_of_edge = colidx.astype(np.int64)
    while it < max_iters:
        # relax the edges of processed tiles against the previous iterate
        new = dist.copy()
        run = active[edge_tile] & (dist[src_of_edge] != INF)
        cand = np.minimum(dist[src_of_edge[run]] + w[run], INF - 1)
        np.minimum.at(new, row_of_edge[run], cand)
        changed = new < dist
        edges.append(int(edges_in_tile[active].sum()))
        it += 1
        dist = new
        if not changed.any():
            ok = True
            break
        # tiles of the next sweep: every tile after a dense sweep, otherwise from each edge out
        # of a changed source to its row's end (a difference array over tile ranges
        # [edge_tile[e], end_tile[row(e)]])
        hit = changed[src_of_edge]
        if sparse is not None and int(hit.sum()) > sparse * T:  # out-degree sum of the changed rows
            active = np.ones(T, dtype=bool)
            continue
        cover = np.zeros(T + 1, dtype=np.int64)
        np.add.at(cover, edge_tile[hit], 1)
        np.add.at(cover, end_tile[row_of_edge[hit]] + 1, -1)
        active = np.cumsum(cover[:T]) > 0
    return dist.astype(np.uint32), it, np.array(edges, dtype=np.int64), ok
