"""Pins for the PageRank oracle (CPU only).

Each check ties the oracle to something other than itself: closed forms on
small graphs, a dense fp64 LU solve, hand-worked sweeps, exact identities
between variants, and the contraction bound of the Jacobi iteration.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2110_01409_gb300.inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cycle(n):
    return I.from_edges(n, np.arange(n), (np.arange(n) + 1) % n, "cycle")


def complete(n):
    s, t = np.meshgrid(np.arange(n), np.arange(n))
    keep = s != t
    return I.from_edges(n, s[keep], t[keep], "complete")


def in_star(k):
    # leaves 1..k -> centre 0; the centre has no out-edges
    return I.from_edges(k + 1, np.arange(1, k + 1), np.zeros(k, dtype=int), "in_star")


def bi_star(k):
    leaves = np.arange(1, k + 1)
    return I.from_edges(k + 1, np.concatenate([leaves, np.zeros(k, int)]),
                        np.concatenate([np.zeros(k, int), leaves]), "bi_star")


ALL_VARIANTS = [
    (oracle.SYNC, 1, 0),
    (oracle.ASYNC, 1, 0),
    (oracle.ASYNC, 3, 0),
    (oracle.DELAYED, 3, 1),
    (oracle.DELAYED, 4, 2),
    (oracle.DELAYED, 2, 1000),
]


@pytest.mark.parametrize("variant,P,delta", ALL_VARIANTS)
@pytest.mark.parametrize("n", [8, 16, 1000])
def test_cycle_is_uniform(variant, P, delta, n):
    # Directed cycle: every M column sums to one and the system is symmetric
    # under rotation, so r = 1/n exactly for every d and every update order.
    g = cycle(n)
    r, it, _, ok = oracle.pagerank(g, variant, d=0.85, tol=1e-12, P=P, delta=delta)
    assert ok
    assert np.max(np.abs(r - 1.0 / n)) < 1e-15


@pytest.mark.parametrize("variant,P,delta", ALL_VARIANTS)
def test_complete_digraph_is_uniform(variant, P, delta):
    g = complete(12)
    r, _, _, ok = oracle.pagerank(g, variant, tol=1e-13, P=P, delta=delta, r0=np.linspace(1, 2, 12) / 18.0)
    assert ok
    assert np.max(np.abs(r - 1.0 / 12)) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 5, 40])
@pytest.mark.parametrize("d", [0.5, 0.85])
def test_in_star_closed_form(k, d):
    # n = k+1; leaves have no in-edges, the centre is dangling:
    # r_leaf = 1/(n + d k), r_centre = (1 + d k)/(n + d k).
    g = in_star(k)
    n = k + 1
    want = np.full(n, 1.0 / (n + d * k))
    want[0] = (1.0 + d * k) / (n + d * k)
    for variant, P, delta in ALL_VARIANTS:
        r, _, _, ok = oracle.pagerank(g, variant, d=d, tol=1e-14, P=P, delta=delta)
        assert ok
        assert np.max(np.abs(r - want)) < 1e-13
    assert np.max(np.abs(oracle.dense_pagerank(g, d) - want)) < 1e-13
    if k == 1 and d == 0.85:
        assert abs(want[1] - 0.350877) < 1e-6 and abs(want[0] - 0.649123) < 1e-6


@pytest.mark.parametrize("k", [1, 3, 17])
def test_bidirectional_star_closed_form(k):
    # r_centre = ((1-d)/n + d)/(1+d), r_leaf = (1 - r_centre)/k
    d, n = 0.85, k + 1
    rc = ((1 - d) / n + d) / (1 + d)
    want = np.full(n, (1 - rc) / k)
    want[0] = rc
    g = bi_star(k)
    r, _, _, ok = oracle.pagerank(g, oracle.SYNC, d=d, tol=1e-14)
    assert ok and np.max(np.abs(r - want)) < 1e-13
    assert np.max(np.abs(oracle.dense_pagerank(g, d) - want)) < 1e-13


def test_ppr_on_cycle_closed_form():
    # teleport e_s on C_n: r_{s+j mod n} = (1-d) d^j / (1 - d^n)
    n, s, d = 16, 5, 0.85
    tele = np.zeros(n)
    tele[s] = 1.0
    want = np.empty(n)
    for j in range(n):
        want[(s + j) % n] = (1 - d) * d**j / (1 - d**n)
    r, _, _, ok = oracle.pagerank(cycle(n), oracle.SYNC, d=d, tol=1e-15, tele=tele)
    assert ok and np.max(np.abs(r - want)) < 1e-14
    r, _, _, ok = oracle.pagerank(cycle(n), oracle.DELAYED, d=d, tol=1e-15, tele=tele, P=3, delta=2)
    assert ok and np.max(np.abs(r - want)) < 1e-14
    assert np.max(np.abs(oracle.dense_pagerank(cycle(n), d, tele) - want)) < 1e-14


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_hand_worked_one_sweep_on_cycle8():
    g = cycle(8)
    r0 = np.zeros(8)
    r0[0] = 1.0
    for row in _golden_rows("cycle8_pagerank_one_sweep.txt"):
        name, P, delta, res = row[0], int(row[1]), int(row[2]), float(row[3])
        want = np.array([float(x) for x in row[4:]])
        if delta < 0:
            r, it, hist, _ = oracle.pagerank(g, oracle.SYNC, d=0.5, tol=0.0, max_iters=1, r0=r0)
        else:
            r, it, hist, _ = oracle.pagerank(g, oracle.DELAYED, d=0.5, tol=0.0, max_iters=1, r0=r0, P=P,
                                             delta=delta, local_read=name.startswith("local"))
        assert it == 1
        assert np.max(np.abs(r - want)) <= 1e-16, name
        assert abs(hist[0] - res) <= 1e-15, name


def _rand_graph(seed, scale=7):
    return I.rmat(scale, 8, seed=seed)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fixed_point_matches_dense_solve(seed):
    g = _rand_graph(seed)
    assert np.any(g.out_degree() == 0), "want dangling vertices in the pin"
    rd = oracle.dense_pagerank(g, 0.85)
    rj = oracle.pagerank_fixed_point(g, 0.85)
    assert np.sum(np.abs(rd - rj)) < 1e-12
    assert abs(rd.sum() - 1.0) < 1e-12
    # weighted + personalized
    w = I.weights_f32(g, seed).astype(np.float64)
    val, s = oracle.normalize(g, w)
    tele = np.zeros(g.n)
    tele[[1, 5, 9]] = 1.0 / 3
    rd = oracle.dense_pagerank(g, 0.85, tele, val)
    rj = oracle.pagerank_fixed_point(g, 0.85, tele, val)
    assert np.sum(np.abs(rd - rj)) < 1e-12


def test_scale10_config_fixed_point_matches_dense():
    g = I.rmat(10, 16, seed=1)
    rd = oracle.dense_pagerank(g, 0.85)
    rj = oracle.pagerank_fixed_point(g, 0.85)
    assert np.sum(np.abs(rd - rj)) < 1e-12


@pytest.mark.parametrize("seed", [4, 5])
def test_p1_extremes_are_gauss_seidel_and_jacobi(seed):
    # Sec. III-B: delta = 0 is the asynchronous algorithm, delta = all of a
    # worker's outputs is the synchronous one. With one worker both are exact.
    g = _rand_graph(seed)
    rs, its, hs, _ = oracle.pagerank(g, oracle.SYNC, tol=1e-10)
    rd, itd, hd, _ = oracle.pagerank(g, oracle.DELAYED, tol=1e-10, P=1, delta=g.n)
    assert its == itd and np.array_equal(rs, rd) and np.array_equal(hs, hd)
    ra, ita, ha, _ = oracle.pagerank(g, oracle.ASYNC, tol=1e-10, P=1)
    rg, itg, hg, _ = oracle.pagerank(g, oracle.DELAYED, tol=1e-10, P=1, delta=0)
    assert ita == itg and np.array_equal(ra, rg)
    # Gauss-Seidel against a plain loop on the same graph (few sweeps, tiny
    # graph); the dangling term is 1 - (mass on vertices with out-edges), read
    # as each row is computed.
    outdeg = g.out_degree()
    r = np.full(g.n, 1.0 / g.n)
    for _ in range(3):
        for v in range(g.n):
            s = sum(r[u] / outdeg[u] for u in g.colidx[g.rowptr[v]:g.rowptr[v + 1]])
            D = 1.0 - r[outdeg > 0].sum()
            r[v] = 0.15 / g.n + 0.85 * (s + D / g.n)
    r3, it3, _, _ = oracle.pagerank(g, oracle.ASYNC, tol=0.0, max_iters=3, P=1)
    assert it3 == 3 and np.max(np.abs(r3 - r)) < 1e-16


def test_equal_blocks_large_delta_is_jacobi():
    # Two equal blocks that both finish on the same tick and flush then: no value
    # crosses blocks within a sweep, so the trajectory is exactly Jacobi.
    g = cycle(64)
    r0 = np.linspace(0.5, 1.5, 64)
    r0 /= r0.sum()
    rs, its, hs, _ = oracle.pagerank(g, oracle.SYNC, tol=1e-9, r0=r0)
    rd, itd, hd, _ = oracle.pagerank(g, oracle.DELAYED, tol=1e-9, r0=r0, P=2, delta=32)
    assert its == itd and np.array_equal(rs, rd)


@pytest.mark.parametrize("seed", [6, 7])
def test_contraction_bound_and_variants_reach_fixed_point(seed):
    g = _rand_graph(seed, scale=9)
    rstar = oracle.dense_pagerank(g, 0.85)
    tol = 1e-6
    r, it, hist, ok = oracle.pagerank(g, oracle.SYNC, tol=tol)
    assert ok and hist[-1] <= tol
    # ||r^k - r*||_1 <= d/(1-d) ||r^k - r^{k-1}||_1
    assert np.sum(np.abs(r - rstar)) <= 0.85 / 0.15 * hist[-1] * (1 + 1e-9)
    # sync iterates keep sum r = 1
    assert abs(r.sum() - 1) < 1e-12
    sync_iters = it
    for P, delta in [(1, 0), (8, 0), (8, 1), (8, 16), (8, 64), (32, 4)]:
        r, it, hist, ok = oracle.pagerank(g, oracle.DELAYED, tol=tol, P=P, delta=delta)
        assert ok
        assert np.sum(np.abs(r - rstar)) < 1e-5
        # fresher values never cost sweeps on this graph (Table I's pattern)
        assert it <= sync_iters


def test_partition_balances_in_degree():
    g = I.rmat(12, 16, seed=3)
    P = 16
    start = oracle.partition(g, P)
    assert start[0] == 0 and start[-1] == g.n and np.all(np.diff(start) >= 0)
    wsum = np.array([(start[p + 1] - start[p]) + g.rowptr[start[p + 1]] - g.rowptr[start[p]] for p in range(P)])
    ideal = (g.n + g.m) / P
    maxrow = np.max(np.diff(g.rowptr)) + 1
    assert np.all(wsum <= ideal + maxrow + 1)


@pytest.mark.parametrize("threads", [2, 4])
def test_threaded_fixed_point_equals_serial_jacobi(threads):
    # the threaded form runs the same synchronous sweeps; only the order of two sums differs
    g = I.rmat(11, 16, seed=9)
    serial = oracle.pagerank_fixed_point(g, 0.85, tol=1e-12)
    par = oracle.pagerank_fixed_point(g, 0.85, tol=1e-12, threads=threads)
    assert np.abs(serial - par).sum() <= 1e-13
    # and it is the dense solve's fixed point
    assert np.abs(par - oracle.dense_pagerank(g, 0.85)).sum() <= 1e-10


def test_threaded_fixed_point_closed_forms():
    # in-star: k leaves -> centre (dangling); r_leaf = 1/(n + d k), r_centre = (1 + d k)/(n + d k)
    k, d = 5, 0.85
    n = k + 1
    g = I.from_edges(n, np.arange(1, n), np.zeros(k, dtype=np.int64))
    r = oracle.pagerank_fixed_point(g, d, tol=1e-15, threads=3)
    assert abs(r[0] - (1 + d * k) / (n + d * k)) <= 1e-13
    assert np.all(np.abs(r[1:] - 1 / (n + d * k)) <= 1e-13)
    # personalized teleport on a directed cycle: r_{s+j} = (1-d) d^j / (1 - d^n)
    n, s = 16, 3
    g = I.from_edges(n, np.arange(n), (np.arange(n) + 1) % n)
    t = np.zeros(n)
    t[s] = 1.0
    r = oracle.pagerank_fixed_point(g, d, tele=t, tol=1e-15, threads=2)
    j = (np.arange(n) - s) % n
    assert np.abs(r - (1 - d) * d ** j / (1 - d ** n)).max() <= 1e-13


def test_row_sweeps_cover_one_sync_sweep():
    # sweeping [0, n) in two row ranges with the whole previous iterate is one synchronous sweep
    g = I.rmat(10, 16, seed=1)
    r0 = np.full(g.n, 1.0 / g.n)
    want, it, hist, _ = oracle.pagerank(g, oracle.SYNC, tol=0.0, max_iters=1, r0=r0)
    out = np.zeros(g.n)
    cut = 400
    a = oracle.pagerank_sweep_rows(g, 0, cut, r0, out)
    b = oracle.pagerank_sweep_rows(g, cut, g.n, r0, out)
    assert np.array_equal(out, want)
    assert a[0] + b[0] == pytest.approx(hist[0], rel=1e-13)
    od = np.bincount(g.colidx, minlength=g.n)
    assert a[1] + b[1] == pytest.approx(want[od > 0].sum(), rel=1e-13)
    # an empty range changes nothing
    assert oracle.pagerank_sweep_rows(g, 5, 5, r0, out) == (0.0, 0.0)
