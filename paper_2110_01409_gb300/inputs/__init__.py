"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

Nothing here computes PageRank or shortest paths: the module draws graphs,
edge weights, source vertices, teleport seed sets and loss weights from
counter-based SplitMix64 draws (see ``graphgen.c``), so the same seed gives the
same bytes on any machine and thread count.

Graphs are returned as in-edge CSR (row ``v`` lists the sources ``u`` of the
edges ``u -> v`` in ascending order), the layout the pull sweep of Sec. III-A
reads. Self-loops and duplicate edges are removed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libdaggen.so")
_lock = threading.Lock()
_lib = None


class _GG(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("m", ctypes.c_int64),
        ("rowptr", ctypes.c_void_p),
        ("colidx", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compiles ``libdaggen.so`` next to its source (host C, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp]
        )
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            p = ctypes.POINTER(_GG)
            lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, p]
            lib.gg_erdos_renyi.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, p]
            lib.gg_banded.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint64, p]
            lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, p]
            lib.gg_take.argtypes = [p, ctypes.c_void_p, ctypes.c_void_p]
            lib.gg_weights_u32.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                           ctypes.c_void_p]
            lib.gg_weights_f32.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                           ctypes.c_void_p]
            lib.gg_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            for f in ("gg_rmat", "gg_erdos_renyi", "gg_banded", "gg_from_edges"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """In-edge CSR: ``colidx[rowptr[v]:rowptr[v+1]]`` are the in-neighbours of ``v``."""

    n: int
    m: int
    rowptr: np.ndarray  # int32 [n+1]
    colidx: np.ndarray  # int32 [m]
    name: str = ""
    meta: dict = field(default_factory=dict)

    def out_degree(self) -> np.ndarray:
        """Number of out-edges of each vertex (its occurrences as an in-neighbour)."""
        return np.bincount(self.colidx, minlength=self.n).astype(np.int32)

    def in_degree(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int32)

    def edges(self):
        """(src, dst) arrays in in-CSR order."""
        dst = np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.rowptr))
        return self.colidx.copy(), dst


def _take(g: _GG, name: str, meta: dict) -> Graph:
    lib = _load()
    rowptr = np.empty(g.n + 1, dtype=np.int32)
    colidx = np.empty(max(g.m, 1), dtype=np.int32)
    lib.gg_take(ctypes.byref(g), rowptr.ctypes.data, colidx.ctypes.data)
    return Graph(int(g.n), int(g.m), rowptr, colidx[: g.m], name, meta)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed (code {rc})")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1) -> Graph:
    """RMAT graph, n = 2^scale, n*edge_factor draws before self-loop/duplicate removal."""
    g = _GG()
    _check(_load().gg_rmat(scale, edge_factor, a, b, c, seed, ctypes.byref(g)), "rmat")
    return _take(g, f"rmat{scale}", dict(scale=scale, edge_factor=edge_factor, a=a, b=b, c=c, seed=seed))


def erdos_renyi(n: int, avg_degree: int = 16, seed: int = 3) -> Graph:
    g = _GG()
    _check(_load().gg_erdos_renyi(n, avg_degree, seed, ctypes.byref(g)), "erdos_renyi")
    return _take(g, f"er{n}", dict(n=n, avg_degree=avg_degree, seed=seed))


def banded(n: int, local: int = 15, band: int = 1024, longrange: int = 1, seed: int = 3) -> Graph:
    g = _GG()
    _check(_load().gg_banded(n, local, band, longrange, seed, ctypes.byref(g)), "banded")
    return _take(g, f"banded{n}", dict(n=n, local=local, band=band, longrange=longrange, seed=seed))


def from_edges(n: int, src, dst, name: str = "edges") -> Graph:
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    g = _GG()
    _check(_load().gg_from_edges(n, src.size, src.ctypes.data, dst.ctypes.data, ctypes.byref(g)), "from_edges")
    return _take(g, name, dict(n=n))


def weights_u32(g: Graph, seed: int) -> np.ndarray:
    """Per-in-edge uint32 weights uniform in [1, 255], keyed by (seed, source, target)."""
    w = np.empty(max(g.m, 1), dtype=np.uint32)
    _load().gg_weights_u32(g.n, g.rowptr.ctypes.data, g.colidx.ctypes.data, seed, w.ctypes.data)
    return w[: g.m]


def weights_f32(g: Graph, seed: int) -> np.ndarray:
    """Per-in-edge float32 weights uniform in (0, 1], keyed by (seed, source, target)."""
    w = np.empty(max(g.m, 1), dtype=np.float32)
    _load().gg_weights_f32(g.n, g.rowptr.ctypes.data, g.colidx.ctypes.data, seed, w.ctypes.data)
    return w[: g.m]


def draws(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` raw uint64 counter-based draws for (seed, stream)."""
    out = np.empty(max(count, 1), dtype=np.uint64)
    _load().gg_draws(seed, stream, count, out.ctypes.data)
    return out[:count]


def _below(h: np.ndarray, k: int) -> np.ndarray:
    return (((h >> np.uint64(32)) * np.uint64(k)) >> np.uint64(32)).astype(np.int64)


def distinct_choice(pool: np.ndarray, k: int, seed: int, stream: int) -> np.ndarray:
    """``k`` distinct elements of ``pool``, drawn uniformly in order of first appearance."""
    if k > len(pool):
        raise ValueError("pool smaller than k")
    out, seen, start = [], set(), 0
    while len(out) < k:
        h = draws(seed, stream, start + 4 * k + 16)[start:]
        start += len(h)
        for i in _below(h, len(pool)):
            x = int(pool[i])
            if x not in seen:
                seen.add(x)
                out.append(x)
                if len(out) == k:
                    break
    return np.array(out, dtype=np.int64)


def sources(g: Graph, k: int, seed: int) -> np.ndarray:
    """``k`` distinct SSSP sources uniform among vertices with out-degree > 0."""
    pool = np.nonzero(g.out_degree() > 0)[0]
    return distinct_choice(pool, k, seed, stream=101).astype(np.uint32)


def ppr_seed_sets(n: int, B: int, seed: int, max_seeds: int = 64):
    """B personalized-PageRank seed sets: each has k ~ U{1..max_seeds} distinct
    vertices drawn uniformly from [0, n). Returns a list of int64 arrays."""
    ks = 1 + _below(draws(seed, 201, B), max_seeds)
    pool = np.arange(n, dtype=np.int64)
    return [distinct_choice(pool, int(ks[c]), seed, stream=1000 + c) for c in range(B)]


def teleport_matrix(n: int, seed_sets) -> np.ndarray:
    """Dense row-major V[n][B] with column c uniform over seed_sets[c]."""
    B = len(seed_sets)
    V = np.zeros((n, B), dtype=np.float32)
    for c, s in enumerate(seed_sets):
        V[s, c] = np.float32(1.0 / len(s))
    return V


def standard_normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Box-Muller standard normals from counter-based uniform draws (float64)."""
    h1 = draws(seed, stream, count)
    h2 = draws(seed, stream + 1, count)
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)  # (0, 1]
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def adjoint_targets(n: int, k: int, seed: int):
    """``k`` distinct uniform target vertices and their loss weights w_i ~ N(0, 1)."""
    t = distinct_choice(np.arange(n, dtype=np.int64), k, seed, stream=301)
    w = standard_normal(seed, 401, k)
    return t, w
