"""CPU oracle for delayed-asynchronous PageRank and Bellman-Ford SSSP.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. It shares
no code with the CUDA path; both read graphs from
``paper_2110_01409_gb300.inputs`` only.

Two parts:

* ``oracle.c`` (built to ``liboracle.so``): fp64 PageRank trajectories of the
  three variants (sync, delayed with P round-robin workers and buffer delta,
  async = delta 0), Bellman-Ford trajectories, Dijkstra, the fp64 PageRank
  adjoint and its gradients, and the paper's OpenMP CPU scheme for timing.
* ``dense.py``: the plain linear-algebra definitions (numpy, fp64) that pin the
  above on small graphs: the PageRank fixed point as a dense solve, the dense
  adjoint, and central finite differences.
* ``frontier.py``: synchronous Bellman-Ford with work skipped where no input
  changed (conditionally processed tiles), counting the edges each sweep
  touches at the GPU's tile granularity.

Parity is pinned for every function here by the tests under ``tests/`` against
closed forms, brute force or a dense solve; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SYNC, ASYNC, DELAYED = 0, 1, 2
INF = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compiles ``liboracle.so`` (plain C, -O2, OpenMP for the timed threaded form)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_SO)
            for f in ("orc_pagerank_sync", "orc_pagerank_delayed", "orc_pagerank_delayed_view", "orc_sssp_sync",
                      "orc_sssp_delayed", "orc_sssp_delayed_view",
                      "orc_dijkstra", "orc_pagerank_adjoint", "orc_pagerank_threads", "orc_sssp_threads",
                      "orc_pagerank_sync_par", "orc_pagerank_sweep_rows"):
                getattr(_lib, f).restype = ctypes.c_int
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _f64(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float64)


def out_degree(g) -> np.ndarray:
    out = np.empty(g.n, dtype=np.int32)
    _load().orc_out_degree(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)), _p(out))
    return out


def partition(g, P: int) -> np.ndarray:
    """Block starts (P+1 values) balanced by in-degree + 1 per vertex (Sec. III-A)."""
    start = np.empty(P + 1, dtype=np.int32)
    _load().orc_partition(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), ctypes.c_int32(P), _p(start))
    return start


def pagerank(g, variant=SYNC, d=0.85, tol=1e-6, max_iters=10000, P=1, delta=0, tele=None, val=None,
             r0=None, local_read=False):
    """fp64 PageRank trajectory. Returns (r, iters, residual history, converged).

    variant SYNC: Jacobi; ASYNC: delayed with delta = 0; DELAYED: P round-robin
    workers with buffer delta (delta = 0 is async). r0 defaults to ``tele`` or 1/n.
    local_read: a worker reads its own unflushed values (Sec. III-C).
    """
    rowptr, colidx = _i32(g.rowptr), _i32(g.colidx)
    tele, val = _f64(tele), _f64(val)
    if r0 is None:
        r = tele.copy() if tele is not None else np.full(g.n, 1.0 / g.n)
    else:
        r = _f64(r0).copy()
    iters = ctypes.c_int32(0)
    hist = np.zeros(max_iters, dtype=np.float64)
    lib = _load()
    if variant == SYNC:
        rc = lib.orc_pagerank_sync(ctypes.c_int32(g.n), _p(rowptr), _p(colidx), _p(val), ctypes.c_double(d),
                                   _p(tele), ctypes.c_double(tol), ctypes.c_int32(max_iters), _p(r),
                                   ctypes.byref(iters), _p(hist))
    else:
        dl = 0 if variant == ASYNC else delta
        rc = lib.orc_pagerank_delayed_view(ctypes.c_int32(g.n), _p(rowptr), _p(colidx), _p(val),
                                           ctypes.c_double(d), _p(tele), ctypes.c_double(tol),
                                           ctypes.c_int32(max_iters), ctypes.c_int32(P), ctypes.c_int32(dl),
                                           ctypes.c_int32(1 if local_read else 0), _p(r), ctypes.byref(iters),
                                           _p(hist))
    if rc < 0:
        raise RuntimeError(f"oracle pagerank failed ({rc})")
    return r, int(iters.value), hist[: iters.value], rc == 0


def pagerank_fixed_point(g, d=0.85, tele=None, val=None, tol=1e-13, max_iters=100000, threads=1):
    """The fixed point r* by fp64 Jacobi to an L1 change <= tol (error <= tol*d/(1-d)).
    threads > 1 computes each sweep's rows on that many OpenMP threads (same iterates)."""
    if threads <= 1:
        r, it, _, ok = pagerank(g, SYNC, d=d, tol=tol, max_iters=max_iters, tele=tele, val=val)
    else:
        tele, val = _f64(tele), _f64(val)
        r = tele.copy() if tele is not None else np.full(g.n, 1.0 / g.n)
        iters = ctypes.c_int32(0)
        rc = _load().orc_pagerank_sync_par(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)), _p(val),
                                           ctypes.c_double(d), _p(tele), ctypes.c_double(tol),
                                           ctypes.c_int32(max_iters), ctypes.c_int32(threads), _p(r),
                                           ctypes.byref(iters))
        if rc < 0:
            raise RuntimeError("oracle fixed point failed")
        ok = rc == 0
    if not ok:
        raise RuntimeError("fixed point did not converge")
    return r


def pagerank_sweep_rows(g, lo, hi, r_in, r_out, d=0.85, tele=None, N=None):
    """One synchronous sweep of rows [lo, hi) into r_out (fp64); N: mass on vertices with out-edges
    of r_in (computed here when not given). Returns (residual over the range, N over the range)."""
    tele = _f64(tele)
    T = 1.0 if tele is None else float(tele.sum())
    if N is None:
        N = float(r_in[out_degree(g) > 0].sum())
    sums = np.zeros(2)
    rc = _load().orc_pagerank_sweep_rows(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)), _p(None),
                                         ctypes.c_double(d), _p(tele), ctypes.c_double(T), ctypes.c_double(N),
                                         ctypes.c_int32(lo), ctypes.c_int32(hi), _p(r_in), _p(r_out), _p(sums))
    if rc != 0:
        raise RuntimeError("oracle row sweep failed")
    return float(sums[0]), float(sums[1])


def sssp_sweep_rows(g, w, lo, hi, d_in, d_out) -> int:
    """One synchronous Bellman-Ford sweep of rows [lo, hi) into d_out (uint32); returns rows lowered."""
    lib = _load()
    lib.orc_sssp_sweep_rows.restype = ctypes.c_int64
    return int(lib.orc_sssp_sweep_rows(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)),
                                       _p(np.ascontiguousarray(w, dtype=np.uint32)), ctypes.c_int32(lo),
                                       ctypes.c_int32(hi), _p(d_in), _p(d_out)))


def sssp(g, w, src, variant=SYNC, P=1, delta=0, max_iters=None, local_read=False):
    """Bellman-Ford trajectory. Returns (dist uint32, iters, updates per sweep, converged)."""
    rowptr, colidx = _i32(g.rowptr), _i32(g.colidx)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    max_iters = g.n + 1 if max_iters is None else max_iters
    dist = np.empty(g.n, dtype=np.uint32)
    iters = ctypes.c_int32(0)
    upd = np.zeros(max_iters, dtype=np.int64)
    lib = _load()
    if variant == SYNC:
        rc = lib.orc_sssp_sync(ctypes.c_int32(g.n), _p(rowptr), _p(colidx), _p(w), ctypes.c_uint32(src),
                               ctypes.c_int32(max_iters), _p(dist), ctypes.byref(iters), _p(upd))
    else:
        dl = 0 if variant == ASYNC else delta
        rc = lib.orc_sssp_delayed_view(ctypes.c_int32(g.n), _p(rowptr), _p(colidx), _p(w), ctypes.c_uint32(src),
                                       ctypes.c_int32(max_iters), ctypes.c_int32(P), ctypes.c_int32(dl),
                                       ctypes.c_int32(1 if local_read else 0), _p(dist), ctypes.byref(iters),
                                       _p(upd))
    if rc < 0:
        raise RuntimeError(f"oracle sssp failed ({rc})")
    return dist, int(iters.value), upd[: iters.value], rc == 0


def dijkstra(g, w, src) -> np.ndarray:
    dist = np.empty(g.n, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    rc = _load().orc_dijkstra(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)), _p(w),
                              ctypes.c_uint32(src), _p(dist))
    if rc != 0:
        raise RuntimeError("oracle dijkstra failed")
    return dist


def normalize(g, w):
    """(val, s): val[e] = w[e] / s[src(e)], s[u] = sum of w over u's out-edges (fp64)."""
    w = _f64(w)
    val = np.empty(g.m, dtype=np.float64)
    s = np.empty(g.n, dtype=np.float64)
    _load().orc_normalize(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)), _p(w), _p(val), _p(s))
    return val, s


def pagerank_adjoint(g, val, c, d=0.85, tol=1e-13, max_iters=100000):
    """fp64 Jacobi solve of lambda = c + d M^T lambda + d g (sum lambda)/n; L1 change <= tol*||c||_1."""
    lam = np.empty(g.n, dtype=np.float64)
    it = ctypes.c_int32(0)
    rc = _load().orc_pagerank_adjoint(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)), _p(_f64(val)),
                                      ctypes.c_double(d), _p(_f64(c)), ctypes.c_double(tol),
                                      ctypes.c_int32(max_iters), _p(lam), ctypes.byref(it))
    if rc != 0:
        raise RuntimeError("oracle adjoint did not converge")
    return lam, int(it.value)


def pagerank_grads(g, val, s, d, r, lam):
    """(grad_w per in-edge, grad_t per vertex) from the forward r and adjoint lambda (fp64)."""
    gw = np.empty(g.m, dtype=np.float64)
    gt = np.empty(g.n, dtype=np.float64)
    _load().orc_pagerank_grads(ctypes.c_int32(g.n), _p(_i32(g.rowptr)), _p(_i32(g.colidx)), _p(_f64(val)),
                               _p(_f64(s)), ctypes.c_double(d), _p(_f64(r)), _p(_f64(lam)), _p(gw), _p(gt))
    return gw, gt


def pagerank_threads(g, variant, d=0.85, tol=1e-6, max_iters=1000, threads=None, delta=0):
    """The paper's OpenMP CPU scheme (FP32 scores). Returns (r float32, iters, seconds, converged)."""
    T = threads or os.cpu_count() or 1
    r = np.empty(g.n, dtype=np.float32)
    it = ctypes.c_int32(0)
    sec = ctypes.c_double(0)
    rc = _load().orc_pagerank_threads(ctypes.c_int32(variant), ctypes.c_int32(g.n), _p(_i32(g.rowptr)),
                                      _p(_i32(g.colidx)), ctypes.c_float(d), ctypes.c_double(tol),
                                      ctypes.c_int32(max_iters), ctypes.c_int32(T), ctypes.c_int32(delta), _p(r),
                                      ctypes.byref(it), ctypes.byref(sec))
    if rc < 0:
        raise RuntimeError("oracle threaded pagerank failed")
    return r, int(it.value), float(sec.value), rc == 0


def sssp_threads(g, w, src, variant, max_iters=None, threads=None, delta=0):
    """The paper's OpenMP CPU scheme for Bellman-Ford. Returns (dist, iters, seconds, converged)."""
    T = threads or os.cpu_count() or 1
    max_iters = g.n + 1 if max_iters is None else max_iters
    dist = np.empty(g.n, dtype=np.uint32)
    it = ctypes.c_int32(0)
    sec = ctypes.c_double(0)
    rc = _load().orc_sssp_threads(ctypes.c_int32(variant), ctypes.c_int32(g.n), _p(_i32(g.rowptr)),
                                  _p(_i32(g.colidx)), _p(np.ascontiguousarray(w, dtype=np.uint32)),
                                  ctypes.c_uint32(src), ctypes.c_int32(max_iters), ctypes.c_int32(T),
                                  ctypes.c_int32(delta), _p(dist), ctypes.byref(it), ctypes.byref(sec))
    if rc < 0:
        raise RuntimeError("oracle threaded sssp failed")
    return dist, int(it.value), float(sec.value), rc == 0


from .dense import dense_pagerank, dense_adjoint, dense_grads, fd_grads  # noqa: E402,F401
