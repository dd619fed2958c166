"""Seeded input generators: determinism and structure (CPU only)."""
import hashlib

import numpy as np

import paper_2110_01409_gb300.inputs as I


def _digest(g):
    h = hashlib.sha256()
    h.update(g.rowptr.tobytes())
    h.update(g.colidx.tobytes())
    return h.hexdigest()


def _check_csr(g):
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.m and len(g.rowptr) == g.n + 1
    assert np.all(np.diff(g.rowptr) >= 0)
    src, dst = g.edges()
    assert np.all(src != dst), "self-loop"
    assert src.min(initial=0) >= 0 and src.max(initial=0) < g.n
    for v in range(0, g.n, max(1, g.n // 257)):
        row = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
        assert np.all(np.diff(row) > 0), "row not strictly ascending (duplicate or unsorted)"


def test_rmat_deterministic_and_wellformed():
    a = I.rmat(10, seed=1)
    b = I.rmat(10, seed=1)
    c = I.rmat(10, seed=2)
    assert _digest(a) == _digest(b)
    assert _digest(a) != _digest(c)
    assert a.n == 1024 and 0 < a.m < 16 * 1024
    _check_csr(a)
    # a = 0.57 > d = 0.05: low ids gather far more edges than high ids
    indeg = a.in_degree()
    assert indeg[:64].sum() > 4 * indeg[-64:].sum()


def test_erdos_renyi_and_banded():
    g = I.erdos_renyi(4096, 16, seed=3)
    _check_csr(g)
    assert 0.97 * 16 * 4096 < g.m <= 16 * 4096
    b = I.banded(8192, local=15, band=1024, longrange=1, seed=3)
    _check_csr(b)
    src, dst = b.edges()
    off = (dst.astype(np.int64) - src) % b.n
    off = np.minimum(off, b.n - off)
    # at most one long-range edge per source lies outside the band
    assert np.sum(off > 1024) <= b.n
    assert np.mean(off <= 1024) > 0.9


def test_from_edges_dedups_and_drops_self_loops():
    g = I.from_edges(4, [0, 0, 1, 2, 2, 3], [1, 1, 1, 3, 0, 3])
    assert g.m == 3
    assert list(g.rowptr) == [0, 1, 2, 2, 3]
    assert list(g.colidx) == [2, 0, 2]


def test_weights_ranges_and_keying():
    g = I.rmat(8, seed=5)
    w = I.weights_u32(g, 7)
    assert w.dtype == np.uint32 and w.min() >= 1 and w.max() <= 255
    f = I.weights_f32(g, 7)
    assert f.dtype == np.float32 and f.min() > 0 and f.max() <= 1
    assert np.array_equal(w, I.weights_u32(g, 7))
    assert not np.array_equal(w, I.weights_u32(g, 8))


def test_sources_seedsets_targets():
    g = I.rmat(10, seed=1)
    s = I.sources(g, 8, seed=2)
    assert len(set(s.tolist())) == 8
    assert np.all(g.out_degree()[s] > 0)
    sets = I.ppr_seed_sets(g.n, 16, seed=4)
    assert all(1 <= len(x) <= 64 and len(set(x.tolist())) == len(x) for x in sets)
    V = I.teleport_matrix(g.n, sets)
    assert np.allclose(V.sum(axis=0), 1.0, atol=1e-6)
    t, w = I.adjoint_targets(g.n, 64, seed=5)
    assert len(set(t.tolist())) == 64
    z = I.standard_normal(9, 11, 20000)
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1) < 0.05
