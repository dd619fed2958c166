"""Autotuner for the sweep's launch choices: variant, delta (Sec. III-B) and
rows per CTA (through the worker cap).

The paper leaves the choice of delta open and notes that it depends on the
platform, the input and the algorithm (Sec. IV, V). This tuner picks it
empirically: it runs complete solves for a small grid of candidates on the
caller's graph and problem and keeps the fastest, measured with the library's
own CUDA-event timing. Results are cached in a JSON file keyed by a graph
fingerprint, so a graph is tuned once per machine. Two tile shapes are in
play: the CTA tiles of the default sweeps (256 threads x 7 items, fixed when
the library is compiled) and the warp tiles of warp-worker sweeps
(reads "warp...", DAG_WARP_WORKERS) and of ordered warp sweeps (reads
"ordered...", DAG_WARP_ORDERED), 32 lanes x 5, 7 or 11 items, which a
candidate's fourth field selects.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

import numpy as np
import torch

from . import dag

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "dag_autotune.json")
_lock = threading.Lock()

# (variant, delta[, reads[, warp tile items per lane]]); reads defaults to "refresh" (see
# dag.READ_MODES), the warp tile to 7 items per lane (used by the "warp..." and "ordered..." read paths only)
SINGLE_CANDIDATES = [("sync", 0), ("async", 0), ("async", 0, "own_l1"), ("async", 0, "cached"), ("delayed", 32),
                     ("delayed", 256), ("delayed", 4096), ("delayed", 4096, "local"),
                     ("sync", 0, "warp"), ("async", 0, "warp+cached"), ("async", 0, "warp+cached", 5),
                     ("async", 0, "warp+cached", 11), ("delayed", 16, "warp"), ("delayed", 256, "warp+cached"),
                     ("async", 0, "ordered+cached", 7), ("async", 0, "ordered+cached", 11)]
WARP_TILES = (5, 7, 11)
SSSP_EXTRA = [("async", 0, "frontier"), ("async", 0, "own_l1+frontier"), ("async", 0, "cached+frontier"),
              ("async", 0, "warp+frontier"), ("async", 0, "warp+cached+frontier"), ("async", 0, "ordered+frontier"),
              ("async", 0, "ordered+cached+frontier")]  # Bellman-Ford only
BATCH_CANDIDATES = [("sync", 0), ("async", 0), ("delayed", 4), ("delayed", 16)]
WORKER_FRACTIONS = [1.0, 0.5]


def fingerprint(plan: dag.Plan) -> str:
    """n, m and a hash of a strided sample of the CSR (device arrays)."""
    n, m = plan.n, plan.m
    rp = plan.rowptr[:: max(1, (n + 1) // 4096)].cpu().numpy()
    ci = plan.colidx[:: max(1, m // 4096)].cpu().numpy() if m else np.zeros(0, np.int32)
    h = hashlib.sha1(rp.tobytes() + ci.tobytes()).hexdigest()[:16]
    return f"n{n}_m{m}_{h}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(path, key, value):
    with _lock:
        data = _load(path)
        data[key] = value
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _norm(c):
    """(variant, delta, reads, warp tile) from a 2-, 3- or 4-tuple candidate."""
    reads = c[2] if len(c) > 2 else "refresh"
    ipt = int(c[3]) if len(c) > 3 else 7
    if ipt not in WARP_TILES:
        raise ValueError(f"warp tile of {ipt} items per lane is not built")
    return (c[0], int(c[1]), reads, ipt)


def _run(plan, algo, variant, delta, reads, kw):
    if algo == "pagerank":
        _, st = dag.pagerank(plan, variant=variant, delta=delta, reads=reads, **kw)
        return st["ms"], st
    if algo == "sssp":
        _, st = dag.sssp(plan, kw["src"], kw["w"], variant=variant, delta=delta, reads=reads)
        return st["ms"], st
    if reads != "refresh":
        raise ValueError("the batched forms take no read mode")
    if algo == "ppr_batched":
        _, _, st = dag.ppr_batched(plan, kw["V"], variant=variant, delta=delta, tol=kw.get("tol", 1e-6))
        return st["ms"], st
    if algo == "sssp_batched":
        _, _, st = dag.sssp_batched(plan, kw["srcs"], kw["w"], variant=variant, delta=delta)
        return st["ms"], st
    raise ValueError(algo)


def tune(plan: dag.Plan, algo: str, candidates=None, worker_fractions=None, trials: int = 2,
         cache: str | None = DEFAULT_CACHE, locality_cutoff: float | None = None, **kw) -> dict:
    """Fastest (variant, delta, workers) for `algo` on this plan's graph.

    algo: "pagerank" (kw: tol, teleport, ...), "sssp" (kw: src, w), "ppr_batched"
    (kw: V), "sssp_batched" (kw: srcs, w). Returns a dict with the choice and the
    measured candidates; leaves the plan's worker cap at the chosen value.

    locality_cutoff: the precomputed-topology signal of Sec. V. The access
    matrix of the full launch's partition is counted first; when the share of
    reads a worker makes of its own block reaches the cutoff, the buffered
    (delayed) candidates are not timed, since buffering does not relieve
    contention on a graph whose updates are read mostly by their writer
    (Sec. IV-C).
    """
    batched = algo.endswith("batched")
    default = BATCH_CANDIDATES if batched else SINGLE_CANDIDATES + (SSSP_EXTRA if algo == "sssp" else [])
    cands = [_norm(c) for c in (candidates or default)]
    fracs = worker_fractions or WORKER_FRACTIONS
    B = int(kw["V"].shape[1]) if algo == "ppr_batched" else (int(kw["srcs"].numel()) if algo == "sssp_batched" else 1)
    key = f"{fingerprint(plan)}|{algo}|B{B}"
    if cache:
        hit = _load(cache).get(key)
        if hit:
            plan.set_worker_cap(hit["workers"])
            if dag.uses_warp_tile(str(hit.get("reads", ""))):
                plan.set_warp_tile(hit.get("warp_tile", 7))
            return hit
    plan.set_worker_cap(0)
    full = plan.workers("async", 0)
    signal = None
    if locality_cutoff is not None:
        signal = dag.locality(dag.access_matrix(plan, full))
        if signal["diag_share"] >= locality_cutoff:
            cands = [c for c in cands if c[0] != "delayed"] or cands
    results = []
    for frac in fracs:
        cap = max(1, int(full * frac))
        plan.set_worker_cap(0 if frac >= 1.0 else cap)
        for variant, delta, reads, ipt in cands:
            times, sweeps = [], []
            try:
                if dag.uses_warp_tile(reads):
                    plan.set_warp_tile(ipt)
                for _ in range(trials):
                    ms, st = _run(plan, algo, variant, delta, reads, kw)
                    times.append(ms)
                    sweeps.append(st.get("iters", st.get("sweeps")))
            except dag.DagError as e:  # e.g. a delta whose buffer cannot be resident
                results.append(dict(variant=variant, delta=delta, reads=reads, warp_tile=ipt,
                                    workers=0 if frac >= 1.0 else cap, error=str(e)))
                continue
            results.append(dict(variant=variant, delta=delta, reads=reads, warp_tile=ipt,
                                workers=0 if frac >= 1.0 else cap, ms=float(np.median(times)), sweeps=sweeps))
    ok = [r for r in results if "ms" in r]
    best = min(ok, key=lambda r: r["ms"])
    choice = dict(variant=best["variant"], delta=best["delta"], reads=best["reads"], warp_tile=best["warp_tile"],
                  workers=best["workers"], ms=best["ms"], candidates=results)
    if signal is not None:
        choice["locality"] = signal
    plan.set_worker_cap(best["workers"])
    if dag.uses_warp_tile(best["reads"]):
        plan.set_warp_tile(best["warp_tile"])
    if cache:
        _store(cache, key, choice)
    torch.cuda.synchronize()
    return choice
