"""Pins for the PageRank adjoint and gradient oracle (CPU only)."""
import numpy as np
import pytest

import oracle
import paper_2110_01409_gb300.inputs as I


def _problem(seed, scale=6):
    g = I.rmat(scale, 8, seed=seed)
    w = I.weights_f32(g, seed).astype(np.float64)
    t = np.zeros(g.n)
    t[[0, 3, 7]] = 1.0 / 3
    targets, wt = I.adjoint_targets(g.n, 8, seed)
    c = np.zeros(g.n)
    c[targets] = wt
    return g, w, t, c


@pytest.mark.parametrize("seed", [1, 2])
def test_dense_gradients_match_finite_differences(seed):
    g, w, t, c = _problem(seed)
    gw, gt, _, _ = oracle.dense_grads(g, w, t, c)
    edges = np.arange(0, g.m, max(1, g.m // 64))
    fw, ft = oracle.fd_grads(g, w, t, c, edges=edges)
    scale = np.max(np.abs(gw[edges]))
    assert np.max(np.abs(fw - gw[edges])) <= 1e-6 * scale
    assert np.max(np.abs(ft - gt)) <= 1e-10 * np.max(np.abs(gt))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_c_adjoint_and_grads_match_dense(seed):
    g, w, t, c = _problem(seed, scale=8)
    val, s = oracle.normalize(g, w)
    lam_d = oracle.dense_adjoint(g, c, 0.85, val)
    lam, it = oracle.pagerank_adjoint(g, val, c, 0.85, tol=1e-14)
    assert np.max(np.abs(lam - lam_d)) <= 1e-11 * np.max(np.abs(lam_d))
    r = oracle.dense_pagerank(g, 0.85, t, val)
    gw, gt = oracle.pagerank_grads(g, val, s, 0.85, r, lam)
    gw_d, gt_d, _, _ = oracle.dense_grads(g, w, t, c)
    assert np.max(np.abs(gw - gw_d)) <= 1e-10 * np.max(np.abs(gw_d))
    assert np.max(np.abs(gt - gt_d)) <= 1e-10 * np.max(np.abs(gt_d))


def test_normalisation_makes_edge_gradients_scale_free():
    # M is unchanged when all out-weights of u are scaled, so
    # sum over u's out-edges of dL/dw_e * w_e = 0 for every u with out-edges.
    g, w, t, c = _problem(4, scale=8)
    gw, _, _, _ = oracle.dense_grads(g, w, t, c)
    acc = np.bincount(g.colidx, weights=gw * w, minlength=g.n)
    ref = np.bincount(g.colidx, weights=np.abs(gw * w), minlength=g.n)
    has_out = np.bincount(g.colidx, minlength=g.n) > 0
    assert np.all(np.abs(acc[has_out]) <= 1e-10 * np.maximum(ref[has_out], 1e-300))


def test_adjoint_with_uniform_weights_is_plain_pagerank_adjoint():
    # all weights equal -> P_vu = 1/outdeg(u), the unweighted matrix
    g, _, t, c = _problem(5, scale=7)
    ones = np.ones(g.m)
    val, _ = oracle.normalize(g, ones)
    lam_w, _ = oracle.pagerank_adjoint(g, val, c, 0.85, tol=1e-14)
    lam_u, _ = oracle.pagerank_adjoint(g, None, c, 0.85, tol=1e-14)
    assert np.max(np.abs(lam_w - lam_u)) <= 1e-12 * np.max(np.abs(lam_u))
    # and the forward fixed point of the same problem solves the transposed system's dual:
    # c^T r = lambda^T (1-d) t
    r = oracle.dense_pagerank(g, 0.85, t)
    assert abs(c @ r - 0.15 * lam_u @ t) <= 1e-12 * max(1.0, abs(c @ r))
