"""Python binding of libdag.so (ctypes): argument marshalling only.

Every step of a solve runs in the CUDA library; this module turns torch CUDA
tensors into device pointers, passes the current torch stream, and turns
status codes into exceptions. Loading fails loudly when libdag.so is missing
(build it with ``paper_2110_01409_gb300.build.build()``): there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdag.so")

OK, ERR_INVALID, ERR_NOT_CONVERGED, ERR_BARRIER_TIMEOUT, ERR_CUDA, ERR_NOMEM = 0, -1, -2, -3, -4, -5
SYNC, ASYNC, DELAYED = 0, 1, 2
VARIANTS = {"sync": SYNC, "async": ASYNC, "delayed": DELAYED}
WARM_START = 1
READ_MODES = {"refresh": 0, "coherent": 2, "cached": 4,  # delayed form's reads (DAG_READ_*); async: cached gathers
              "local": 8, "local+coherent": 10, "local+cached": 12,
              "own_l1": 16,  # async form: own block through L1 (DAG_READ_OWN_L1)
              "frontier": 32, "own_l1+frontier": 48,  # Bellman-Ford: run only changed tiles (DAG_SSSP_FRONTIER)
              "cached+frontier": 36,
              "warp": 64, "warp+coherent": 66, "warp+cached": 68,  # one worker per warp (DAG_WARP_WORKERS)
              "warp+frontier": 96, "warp+cached+frontier": 100,  # async Bellman-Ford: warp-tile frontier
              "ordered+frontier": 160, "ordered+cached+frontier": 164,  # ... dense sweeps on CTA-ordered tiles
              "ordered": 128, "ordered+cached": 132}  # async: warps take the path's tiles in turn (DAG_WARP_ORDERED)


def uses_warp_tile(reads: str) -> bool:
    """True for the read paths that run warp tiles (Plan.set_warp_tile selects their shape)."""
    return reads.startswith(("warp", "ordered"))

EXPORTS = (
    "dag_plan_create", "dag_plan_destroy", "dag_plan_out_degree", "dag_partition", "dag_workers",
    "dag_pagerank", "dag_sssp", "dag_ppr_batched", "dag_sssp_batched", "dag_transpose",
    "dag_normalize_weights", "dag_pagerank_adjoint", "dag_strerror", "dag_last_error_message",
    "dag_debug_skip_barrier_once", "dag_debug_stall_staging_once", "dag_tile_items", "dag_pagerank_noalloc", "dag_gather_f32", "dag_plan_set_worker_cap",
    "dag_sssp_u8", "dag_probe_gather", "dag_access_matrix", "dag_plan_set_batched_graph", "dag_warp_tile_items",
    "dag_plan_set_warp_tile", "dag_plan_last_status", "dag_sssp_batched_u8", "dag_rank_to_state",
    "dag_state_to_rank", "dag_pagerank_sweep_rows", "dag_sssp_sweep_rows", "dag_plan_set_warp_frontier_marks",
    "dag_plan_set_batched_wide",
)


class DagError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("d_rowptr", ctypes.c_void_p),
                ("d_colidx", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("err", ctypes.c_int32), ("residual", ctypes.c_double),
                ("ms", ctypes.c_float), ("workers", ctypes.c_int32), ("delta", ctypes.c_int32),
                ("flushes", ctypes.c_int64), ("edges_processed", ctypes.c_int64)]


class _BStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("err", ctypes.c_int32), ("ms", ctypes.c_float),
                ("workers", ctypes.c_int32), ("delta", ctypes.c_int32), ("column_sweeps", ctypes.c_int64),
                ("graph", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()
_vp, _i32, _f32, _f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, ctypes.c_double


def lib():
    """The loaded libdag.so. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libdag.so not found at {LIB_PATH}; run paper_2110_01409_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            L.dag_plan_create.argtypes = [ctypes.POINTER(_Csr), _i32, ctypes.POINTER(_vp)]
            L.dag_plan_destroy.argtypes = [_vp]
            L.dag_plan_out_degree.argtypes = [_vp, _vp, _vp]
            L.dag_partition.argtypes = [_vp, _i32, _vp]
            L.dag_workers.argtypes = [_vp, _i32, _i32, ctypes.POINTER(_i32)]
            L.dag_pagerank.argtypes = [_vp, _f32, _f64, _i32, _i32, _i32, _vp, _vp, _vp, _i32,
                                       ctypes.POINTER(_Stats), _vp]
            L.dag_sssp.argtypes = [_vp, ctypes.c_uint32, _i32, _i32, _i32, _vp, _vp, _i32, ctypes.POINTER(_Stats),
                                   _vp]
            L.dag_ppr_batched.argtypes = [_vp, _f32, _f64, _i32, _i32, _i32, _i32, _vp, _vp, _vp,
                                          ctypes.POINTER(_BStats), _vp]
            L.dag_sssp_batched.argtypes = [_vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp,
                                           ctypes.POINTER(_BStats), _vp]
            L.dag_sssp_batched_u8.argtypes = [_vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp,
                                              ctypes.POINTER(_BStats), _vp]
            L.dag_transpose.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.dag_normalize_weights.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.dag_pagerank_adjoint.argtypes = [_vp, _vp, _f32, _f64, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp,
                                               _vp, _vp, _vp, _i32, ctypes.POINTER(_Stats), _vp]
            L.dag_strerror.argtypes = [_i32]
            L.dag_strerror.restype = ctypes.c_char_p
            L.dag_last_error_message.argtypes = []
            L.dag_last_error_message.restype = ctypes.c_char_p
            L.dag_debug_skip_barrier_once.argtypes = [_vp, _i32]
            L.dag_debug_stall_staging_once.argtypes = [_vp, _i32]
            L.dag_tile_items.restype = _i32
            L.dag_warp_tile_items.restype = _i32
            L.dag_warp_tile_items.argtypes = [_vp]
            L.dag_plan_set_warp_tile.argtypes = [_vp, _i32]
            L.dag_plan_set_warp_frontier_marks.argtypes = [_vp, _f32]
            L.dag_plan_last_status.argtypes = [_vp, _vp, _vp]
            L.dag_rank_to_state.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.dag_state_to_rank.argtypes = [_vp, _vp, _vp, _vp]
            L.dag_pagerank_sweep_rows.argtypes = [_vp, _f32, _i32, _i32, _vp, _f64, _f64, _vp, _vp, _vp, _vp]
            L.dag_sssp_sweep_rows.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp]
            L.dag_gather_f32.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
            L.dag_plan_set_worker_cap.argtypes = [_vp, _i32]
            L.dag_plan_set_batched_graph.argtypes = [_vp, _i32]
            L.dag_plan_set_batched_wide.argtypes = [_vp, _i32]
            L.dag_access_matrix.argtypes = [_vp, _i32, _vp, _vp]
            L.dag_probe_gather.argtypes = [_vp, ctypes.c_int64, _vp, _i32, _i32, _i32, ctypes.POINTER(_f32), _vp]
            L.dag_sssp_u8.argtypes = [_vp, ctypes.c_uint32, _i32, _i32, _i32, _vp, _vp, _i32,
                                      ctypes.POINTER(_Stats), _vp]
            L.dag_pagerank_noalloc.argtypes = [ctypes.POINTER(_Csr), _f32, _f64, _i32, _i32, _i32, _vp, _vp,
                                               ctypes.POINTER(_Stats), _vp]
            for f in EXPORTS:
                if f not in ("dag_strerror", "dag_last_error_message", "dag_tile_items", "dag_warp_tile_items"):
                    getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _raise(rc: int, allow_not_converged: bool = True):
    if rc == OK or (allow_not_converged and rc == ERR_NOT_CONVERGED):
        return
    L = lib()
    raise DagError(rc, f"{L.dag_strerror(rc).decode()}: {L.dag_last_error_message().decode()}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, n, name):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor of {n} elements")
    return t


def _variant(v):
    return VARIANTS[v] if isinstance(v, str) else int(v)


def _stats(st: _Stats, m: int) -> dict:
    return dict(iters=st.iters, err=st.err, converged=st.err == OK, residual=st.residual, ms=st.ms,
                workers=st.workers, delta=st.delta, flushes=st.flushes, edges_processed=st.edges_processed)


class Plan:
    """Per-graph plan over device CSR tensors (kept alive by the plan)."""

    def __init__(self, rowptr: torch.Tensor, colidx: torch.Tensor, barrier_timeout_ms: int = 0):
        n = rowptr.numel() - 1
        m = colidx.numel()
        _dev(rowptr, torch.int32, n + 1, "rowptr")
        if m:
            _dev(colidx, torch.int32, m, "colidx")
        self.rowptr, self.colidx, self.n, self.m = rowptr, colidx, n, m
        csr = _Csr(n, m, rowptr.data_ptr(), colidx.data_ptr() if m else 0)
        h = ctypes.c_void_p()
        _raise(lib().dag_plan_create(ctypes.byref(csr), barrier_timeout_ms, ctypes.byref(h)), False)
        self.h = h

    @classmethod
    def from_graph(cls, g, device="cuda", **kw):
        rp = torch.from_numpy(g.rowptr).to(device)
        ci = torch.from_numpy(g.colidx).to(device) if g.m else torch.zeros(1, dtype=torch.int32, device=device)[:0]
        return cls(rp, ci, **kw)

    def close(self):
        if getattr(self, "h", None):
            lib().dag_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def out_degree(self) -> torch.Tensor:
        out = torch.empty(self.n, dtype=torch.int32, device=self.rowptr.device)
        _raise(lib().dag_plan_out_degree(self.h, _ptr(out), _stream()), False)
        return out

    def partition(self, workers: int):
        import numpy as np
        start = np.empty(workers + 1, dtype=np.int32)
        _raise(lib().dag_partition(self.h, workers, start.ctypes.data), False)
        return start

    def workers(self, variant="delayed", delta=256) -> int:
        w = _i32(0)
        _raise(lib().dag_workers(self.h, _variant(variant), delta, ctypes.byref(w)), False)
        return w.value

    def set_batched_graph(self, on: bool):
        """Batched solves on this plan through CUDA graphs captured once per launch shape (on, the
        default), or launched directly (off)."""
        _raise(lib().dag_plan_set_batched_graph(self.h, 1 if on else 0), False)

    def set_batched_wide(self, on: bool):
        """Batched sync / async solves of 32, 64, 128 or 256 columns on the wide kernel (a warp per
        share of a tile, all columns; on, the default) or on 32-column warps (off)."""
        _raise(lib().dag_plan_set_batched_wide(self.h, 1 if on else 0), False)

    def set_warp_tile(self, items_per_lane: int):
        """Warp tile shape (32 x items_per_lane items, 5, 7 or 11) of warp-worker solves."""
        _raise(lib().dag_plan_set_warp_tile(self.h, items_per_lane), False)

    def set_warp_frontier_marks(self, marks_per_tile: float):
        """Warp-tile frontier: marks per warp tile at or below which the next sweep runs only stamped tiles."""
        _raise(lib().dag_plan_set_warp_frontier_marks(self.h, float(marks_per_tile)), False)

    def warp_tile_items(self) -> int:
        return int(lib().dag_warp_tile_items(self.h))

    def last_status_to(self, out: torch.Tensor, stream=None):
        """Enqueues a copy of the last solve's (err, converged, sweeps) into out (CUDA int32 [3]); no wait."""
        _dev(out, torch.int32, 3, "out")
        _raise(lib().dag_plan_last_status(self.h, _ptr(out), _stream(stream)), False)

    def set_worker_cap(self, max_workers: int):
        """At most max_workers CTAs per solve (0: as many as fit)."""
        _raise(lib().dag_plan_set_worker_cap(self.h, max_workers), False)

    def debug_skip_barrier_once(self, timeout_ms: int):
        _raise(lib().dag_debug_skip_barrier_once(self.h, timeout_ms), False)

    def debug_stall_staging_once(self, timeout_ms: int):
        _raise(lib().dag_debug_stall_staging_once(self.h, timeout_ms), False)


def pagerank(plan: Plan, d=0.85, tol=1e-6, variant="delayed", delta=256, max_iters=1000, teleport=None,
             val=None, out=None, warm_start=False, stream=None, stats=True, reads="refresh"):
    """PageRank through dag_pagerank. Returns (rank float32 tensor, stats dict or None)."""
    dev = plan.rowptr.device
    out = out if out is not None else torch.empty(plan.n, dtype=torch.float32, device=dev)
    _dev(out, torch.float32, plan.n, "out")
    _dev(teleport, torch.float32, plan.n, "teleport")
    _dev(val, torch.float32, plan.m, "val")
    st = _Stats()
    rc = lib().dag_pagerank(plan.h, d, tol, _variant(variant), delta, max_iters, _ptr(teleport), _ptr(val),
                            _ptr(out), (WARM_START if warm_start else 0) | READ_MODES[reads],
                            ctypes.byref(st) if stats else None,
                            _stream(stream))
    _raise(rc)
    return out, (_stats(st, plan.m) if stats else None)


def sssp(plan: Plan, src: int, w, variant="delayed", delta=32, max_iters=None, out=None, stream=None,
         stats=True, reads="refresh"):
    """Bellman-Ford through dag_sssp (w: int32 view of uint32 weights) or
    dag_sssp_u8 (w: uint8 weights). Returns (dist as int32 holding uint32 bits, stats)."""
    dev = plan.rowptr.device
    out = out if out is not None else torch.empty(plan.n, dtype=torch.int32, device=dev)
    _dev(out, torch.int32, plan.n, "out")
    u8 = w is not None and w.dtype == torch.uint8
    if plan.m:
        _dev(w, torch.uint8 if u8 else torch.int32, plan.m, "w")
    max_iters = plan.n + 1 if max_iters is None else max_iters
    st = _Stats()
    fn = lib().dag_sssp_u8 if u8 else lib().dag_sssp
    rc = fn(plan.h, src, _variant(variant), delta, max_iters, _ptr(w) if plan.m else None, _ptr(out),
            READ_MODES[reads], ctypes.byref(st) if stats else None, _stream(stream))
    _raise(rc)
    return out, (_stats(st, plan.m) if stats else None)


def _bstats(st: _BStats) -> dict:
    return dict(sweeps=st.sweeps, err=st.err, converged=st.err == OK, ms=st.ms, workers=st.workers,
                delta=st.delta, column_sweeps=st.column_sweeps, graph=bool(st.graph))


def ppr_batched(plan: Plan, V: torch.Tensor, d=0.85, tol=1e-6, variant="async", delta=0, max_iters=1000,
                out=None, stream=None, stats=True):
    """B personalized PageRanks; V row-major [n, B]. Returns (R [n, B], iters [B], stats)."""
    n, B = V.shape
    _dev(V, torch.float32, n * B, "V")
    out = out if out is not None else torch.empty_like(V)
    _dev(out, torch.float32, n * B, "out")
    iters = torch.empty(B, dtype=torch.int32, device=V.device)
    st = _BStats()
    rc = lib().dag_ppr_batched(plan.h, d, tol, _variant(variant), delta, max_iters, B, _ptr(V), _ptr(out),
                               _ptr(iters), ctypes.byref(st) if stats else None, _stream(stream))
    _raise(rc)
    return out, iters, (_bstats(st) if stats else None)


def sssp_batched(plan: Plan, srcs: torch.Tensor, w, variant="async", delta=0, max_iters=None, out=None,
                 stream=None, stats=True):
    """B Bellman-Ford solves; srcs int32 [B]; w: int32 view of uint32 weights (dag_sssp_batched) or uint8
    weights (dag_sssp_batched_u8). Returns (D int32 [n, B] holding uint32 bits, iters, stats)."""
    B = srcs.numel()
    _dev(srcs, torch.int32, B, "srcs")
    u8 = w is not None and w.dtype == torch.uint8
    if plan.m:
        _dev(w, torch.uint8 if u8 else torch.int32, plan.m, "w")
    out = out if out is not None else torch.empty((plan.n, B), dtype=torch.int32, device=srcs.device)
    _dev(out, torch.int32, plan.n * B, "out")
    iters = torch.empty(B, dtype=torch.int32, device=srcs.device)
    max_iters = plan.n + 1 if max_iters is None else max_iters
    st = _BStats()
    fn = lib().dag_sssp_batched_u8 if u8 else lib().dag_sssp_batched
    rc = fn(plan.h, _variant(variant), delta, max_iters, B, _ptr(srcs),
                                _ptr(w) if plan.m else None, _ptr(out), _ptr(iters),
                                ctypes.byref(st) if stats else None, _stream(stream))
    _raise(rc)
    return out, iters, (_bstats(st) if stats else None)


def transpose(plan: Plan):
    """Out-edge CSR (rowptr, colidx) and perm: out-edge k is in-edge perm[k]."""
    dev = plan.rowptr.device
    orow = torch.empty(plan.n + 1, dtype=torch.int32, device=dev)
    ocol = torch.empty(max(plan.m, 1), dtype=torch.int32, device=dev)
    perm = torch.empty(max(plan.m, 1), dtype=torch.int32, device=dev)
    _raise(lib().dag_transpose(plan.h, _ptr(orow), _ptr(ocol), _ptr(perm), _stream()), False)
    return orow, ocol[: plan.m], perm[: plan.m]


def normalize_weights(plan: Plan, w: torch.Tensor):
    """(val per in-edge, s per vertex) with val[e] = w[e] / s[src(e)]."""
    _dev(w, torch.float32, plan.m, "w")
    val = torch.empty_like(w)
    s = torch.empty(plan.n, dtype=torch.float32, device=w.device)
    _raise(lib().dag_normalize_weights(plan.h, _ptr(w), _ptr(val), _ptr(s), _stream()), False)
    return val, s


def pagerank_adjoint(in_plan: Plan, out_plan: Plan, val, val_out, s, rank, c, d=0.85, tol=1e-6,
                     variant="delayed", delta=256, max_iters=10000, want_lambda=False, stream=None, reads="refresh"):
    """Adjoint solve + gradients (reads: the adjoint sweep's read path, see READ_MODES; the warp forms run
    on out_plan's warp tile). Returns (grad_w [m], grad_t [n], lambda or None, stats)."""
    n, m = in_plan.n, in_plan.m
    for t, nm in ((rank, "rank"), (s, "s"), (c, "c")):
        if t is None:
            raise ValueError(f"{nm}: required")
        _dev(t, torch.float32, n, nm)
    if m:
        for t, nm in ((val, "val"), (val_out, "val_out")):
            if t is None:
                raise ValueError(f"{nm}: required")
            _dev(t, torch.float32, m, nm)
    dev = rank.device
    gw = torch.empty(in_plan.m, dtype=torch.float32, device=dev)
    gt = torch.empty(in_plan.n, dtype=torch.float32, device=dev)
    lam = torch.empty(in_plan.n, dtype=torch.float32, device=dev) if want_lambda else None
    st = _Stats()
    rc = lib().dag_pagerank_adjoint(in_plan.h, out_plan.h, d, tol, _variant(variant), delta, max_iters,
                                    _ptr(val), _ptr(val_out), _ptr(s), _ptr(rank), _ptr(c), _ptr(gw), _ptr(gt),
                                    _ptr(lam), READ_MODES[reads], ctypes.byref(st), _stream(stream))
    _raise(rc)
    return gw, gt, lam, _stats(st, in_plan.m)


def pagerank_noalloc(rowptr: torch.Tensor, colidx: torch.Tensor, d=0.85, tol=1e-6, variant="delayed", delta=256,
                     max_iters=1000, teleport=None, out=None, stream=None):
    """PageRank through dag_pagerank_noalloc: no plan and no device allocation
    inside the library (n <= 2^20, m <= 2^24). Returns (rank, stats)."""
    n, m = rowptr.numel() - 1, colidx.numel()
    _dev(rowptr, torch.int32, n + 1, "rowptr")
    if m:
        _dev(colidx, torch.int32, m, "colidx")
    out = out if out is not None else torch.empty(n, dtype=torch.float32, device=rowptr.device)
    _dev(out, torch.float32, n, "out")
    _dev(teleport, torch.float32, n, "teleport")
    csr = _Csr(n, m, rowptr.data_ptr(), colidx.data_ptr() if m else 0)
    st = _Stats()
    rc = lib().dag_pagerank_noalloc(ctypes.byref(csr), d, tol, _variant(variant), delta, max_iters, _ptr(teleport),
                                    _ptr(out), ctypes.byref(st), _stream(stream))
    _raise(rc)
    return out, _stats(st, m)


def access_matrix(plan: Plan, workers: int = 32) -> torch.Tensor:
    """[workers, workers] int64: reads by block i (row owner) of block j's vertices (Fig. 5)."""
    out = torch.empty((workers, workers), dtype=torch.int64, device=plan.rowptr.device)
    _raise(lib().dag_access_matrix(plan.h, workers, _ptr(out), _stream()), False)
    return out


def tile_items() -> int:
    """Items (rows + in-edges) per merge-path tile of the sweeps."""
    return int(lib().dag_tile_items())


def locality(counts: torch.Tensor) -> dict:
    """Summary of an access matrix (Fig. 5): the share of all reads that fall on
    the reader's own block (the diagonal), and the rows whose own share is at
    least 1/P (the boxes the paper marks)."""
    c = counts.to(torch.float64)
    P = c.shape[0]
    diag = torch.diagonal(c)
    rows = c.sum(1)
    own = torch.where(rows > 0, diag / rows.clamp_min(1), torch.zeros_like(diag))
    total = float(rows.sum())
    return {"workers": P, "diag_share": float(diag.sum()) / total if total else 0.0,
            "marked_rows": int((own >= 1.0 / P).sum()), "own_share_median": float(own.median())}


def probe_gather(plan: Plan, x: torch.Tensor, coherent=True, repeats=5, stream=None) -> float:
    """ms of one streamed gather pass x[colidx[e]] over the plan's graph (dag_probe_gather)."""
    _dev(x, torch.float32, plan.n, "x")
    ms = _f32(0)
    _raise(lib().dag_probe_gather(_ptr(plan.colidx), plan.m, _ptr(x), plan.n, 1 if coherent else 0, repeats,
                                  ctypes.byref(ms), _stream(stream)), False)
    return ms.value


class WeightedPageRank:
    """Forward/backward of weighted PageRank over one graph: holds the in-edge
    plan, the out-edge CSR and its plan, and the in->out edge permutation."""

    def __init__(self, plan: Plan, d=0.85, tol=1e-6, variant="delayed", delta=256, max_iters=10000,
                 reads="refresh", adjoint_reads=None):
        self.plan, self.d, self.tol, self.variant, self.delta, self.max_iters = plan, d, tol, variant, delta, max_iters
        self.reads = reads
        self.adjoint_reads = reads if adjoint_reads is None else adjoint_reads
        orow, ocol, perm = transpose(plan)
        self.perm = perm
        self.out_plan = Plan(orow, ocol)
        self.out_plan.set_warp_tile(plan.warp_tile_items() // 32)

    def forward(self, w: torch.Tensor, teleport: torch.Tensor | None = None):
        val, s = normalize_weights(self.plan, w)
        r, st = pagerank(self.plan, self.d, self.tol, self.variant, self.delta, self.max_iters, teleport=teleport,
                         val=val, reads=self.reads)
        return r, val, s, st

    def backward(self, val, s, r, c):
        _dev(val, torch.float32, self.plan.m, "val")
        val_out = torch.empty_like(val)
        _raise(lib().dag_gather_f32(_ptr(val), _ptr(self.perm), self.plan.m, _ptr(val_out), _stream()), False)
        return pagerank_adjoint(self.plan, self.out_plan, val, val_out, s, r, c.contiguous(), self.d, self.tol,
                                self.variant, self.delta, self.max_iters, reads=self.adjoint_reads)


class PageRankFn(torch.autograd.Function):
    """r = PageRank(row-normalised w, teleport t); gradients w.r.t. w and t by
    the adjoint sweep (no iterates stored)."""

    @staticmethod
    def forward(ctx, w, t, model: WeightedPageRank):
        r, val, s, st = model.forward(w.detach().contiguous(), None if t is None else t.detach().contiguous())
        ctx.model = model
        ctx.has_t = t is not None
        ctx.save_for_backward(val, s, r)
        ctx.stats = st
        return r

    @staticmethod
    def backward(ctx, grad_r):
        val, s, r = ctx.saved_tensors
        gw, gt, _, st = ctx.model.backward(val, s, r, grad_r.contiguous().float())
        ctx.backward_stats = st
        return gw, (gt if ctx.has_t else None), None


def rank_to_state(plan: Plan, r: torch.Tensor, x: torch.Tensor, linked: torch.Tensor | None = None):
    """x = r / outdeg (r on vertices without out-edges); linked (CUDA float64 [1]) gets sum r over
    vertices with out-edges."""
    _dev(r, torch.float32, plan.n, "r")
    _dev(x, torch.float32, plan.n, "x")
    _dev(linked, torch.float64, 1, "linked")
    _raise(lib().dag_rank_to_state(plan.h, _ptr(r), _ptr(x), _ptr(linked), _stream()), False)


def state_to_rank(plan: Plan, x: torch.Tensor, r: torch.Tensor):
    _dev(x, torch.float32, plan.n, "x")
    _dev(r, torch.float32, plan.n, "r")
    _raise(lib().dag_state_to_rank(plan.h, _ptr(x), _ptr(r), _stream()), False)


def pagerank_sweep_rows(plan: Plan, lo: int, hi: int, x_in, x_out, sums, d=0.85, teleport=None,
                        teleport_total=1.0, linked_mass=0.0):
    """One synchronous PageRank sweep of rows [lo, hi) (dag_pagerank_sweep_rows); sums: CUDA float64 [2]."""
    for t, nm in ((x_in, "x_in"), (x_out, "x_out")):
        _dev(t, torch.float32, plan.n, nm)
    _dev(sums, torch.float64, 2, "sums")
    _dev(teleport, torch.float32, plan.n, "teleport")
    _raise(lib().dag_pagerank_sweep_rows(plan.h, d, lo, hi, _ptr(teleport), teleport_total, linked_mass,
                                         _ptr(x_in), _ptr(x_out), _ptr(sums), _stream()), False)


def sssp_sweep_rows(plan: Plan, lo: int, hi: int, w8, dist_in, dist_out, sums):
    """One synchronous Bellman-Ford sweep of rows [lo, hi) (dag_sssp_sweep_rows); sums: CUDA float64 [2]."""
    for t, nm in ((dist_in, "dist_in"), (dist_out, "dist_out")):
        _dev(t, torch.int32, plan.n, nm)
    if plan.m:
        _dev(w8, torch.uint8, plan.m, "w8")
    _dev(sums, torch.float64, 2, "sums")
    _raise(lib().dag_sssp_sweep_rows(plan.h, lo, hi, _ptr(w8), _ptr(dist_in), _ptr(dist_out), _ptr(sums),
                                     _stream()), False)
