"""Dense fp64 definitions (numpy) that pin the C oracle on small graphs.

TEST INFRASTRUCTURE (see the package docstring).

PageRank as a linear system. The paper states PageRank only in words (Sec. IV-A:
each score is a weighted combination of its in-neighbours' scores); the reading
used throughout is

    r = d (M r + u g^T r) + (1 - d) t,

M_vu = 1/outdeg(u) (or P_vu = w_uv / s_u when weighted), g the indicator of
vertices with no out-edges, u = 1/n (dangling mass spread uniformly) and t the
teleport vector. Its unique solution solves (I - A) r = (1 - d) t with
A = d (M + u g^T). A loss L = c^T r has gradient lambda = (I - A)^{-T} c.
"""
from __future__ import annotations

import numpy as np


def _dense_M(g, val=None):
    n = g.n
    M = np.zeros((n, n), dtype=np.float64)
    outdeg = np.bincount(g.colidx, minlength=n)
    for v in range(n):
        for e in range(g.rowptr[v], g.rowptr[v + 1]):
            u = g.colidx[e]
            M[v, u] += val[e] if val is not None else 1.0 / outdeg[u]
    return M, outdeg


def system_matrix(g, d=0.85, val=None):
    """A = d (M + (1/n) 1 g^T) as a dense fp64 matrix."""
    M, outdeg = _dense_M(g, val)
    gvec = (outdeg == 0).astype(np.float64)
    return d * (M + np.outer(np.full(g.n, 1.0 / g.n), gvec))


def dense_pagerank(g, d=0.85, tele=None, val=None):
    """The PageRank fixed point by a dense LU solve of (I - A) r = (1 - d) t."""
    n = g.n
    t = np.full(n, 1.0 / n) if tele is None else np.asarray(tele, dtype=np.float64)
    A = system_matrix(g, d, val)
    return np.linalg.solve(np.eye(n) - A, (1.0 - d) * t)


def dense_adjoint(g, c, d=0.85, val=None):
    """lambda = (I - A)^{-T} c."""
    A = system_matrix(g, d, val)
    return np.linalg.solve((np.eye(g.n) - A).T, np.asarray(c, dtype=np.float64))


def _normalize(g, w):
    s = np.bincount(g.colidx, weights=w, minlength=g.n).astype(np.float64)
    val = w / s[g.colidx]
    return val, s


def loss(g, w, tele, c, d=0.85):
    """L(w, t) = c^T r(w, t) with r the weighted PageRank of row-normalised w."""
    val, _ = _normalize(g, np.asarray(w, dtype=np.float64))
    return float(np.dot(c, dense_pagerank(g, d, tele, val)))


def dense_grads(g, w, tele, c, d=0.85):
    """Analytic gradients of L = c^T r w.r.t. raw edge weights w (in-CSR order) and t.

    From dL = lambda^T dA r with A = d (M + u g^T): dL/dM_vu = d lambda_v r_u and,
    through M_vu = w_uv / s_u, dL/dw_uv = d r_u (lambda_v - sum_v' M_v'u lambda_v') / s_u;
    dL/dt = (1 - d) lambda.
    """
    w = np.asarray(w, dtype=np.float64)
    val, s = _normalize(g, w)
    r = dense_pagerank(g, d, tele, val)
    lam = dense_adjoint(g, c, d, val)
    M, _ = _dense_M(g, val)
    mt = M.T @ lam
    src = g.colidx
    dst = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    gw = d * r[src] * (lam[dst] - mt[src]) / s[src]
    gt = (1.0 - d) * lam
    return gw, gt, r, lam


def fd_grads(g, w, tele, c, d=0.85, edges=None, rel_h=1e-6):
    """Central finite differences of L w.r.t. the listed edge weights and all of t (fp64).

    h = rel_h * w_e for an edge. L is linear in t, so its teleport gradient is
    taken from one factorisation of (I - A)^T with a step of 1 per entry.
    """
    w = np.asarray(w, dtype=np.float64)
    n = g.n
    t = np.full(n, 1.0 / n) if tele is None else np.asarray(tele, dtype=np.float64)
    edges = np.arange(g.m) if edges is None else np.asarray(edges)
    gw = np.empty(len(edges), dtype=np.float64)
    for k, e in enumerate(edges):
        h = rel_h * w[e]
        wp = w.copy(); wp[e] += h
        wm = w.copy(); wm[e] -= h
        gw[k] = (loss(g, wp, t, c, d) - loss(g, wm, t, c, d)) / (2.0 * h)
    val, _ = _normalize(g, w)
    A = system_matrix(g, d, val)
    Kinv = np.linalg.inv(np.eye(n) - A)
    # L(t + e_v) - L(t - e_v) over 2 = (1 - d) c^T K^{-1} e_v for each v, all at once
    gt = (1.0 - d) * (c @ Kinv)
    return gw, gt
