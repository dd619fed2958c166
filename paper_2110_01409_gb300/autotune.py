"""Autotuner for the sweep's launch choices: variant, delta (Sec. III-B) and
rows per CTA (through the worker cap).

The paper leaves the choice of delta open and notes that it depends on the
platform, the input and the algorithm (Sec. IV, V). This tuner picks it
empirically: it runs complete solves for a small grid of candidates on the
caller's graph and problem and keeps the fastest, measured with the library's
own CUDA-event timing. Results are cached in a JSON file keyed by a graph
fingerprint, so a graph is tuned once per machine. The tile shape (items per
merge-path tile) is fixed when the library is compiled; the grid of launch
shapes measured for it is recorded in the design doc.
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

SINGLE_CANDIDATES = [("sync", 0), ("async", 0), ("delayed", 32), ("delayed", 256), ("delayed", 4096)]
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


def _run(plan, algo, variant, delta, kw):
    if algo == "pagerank":
        _, st = dag.pagerank(plan, variant=variant, delta=delta, **kw)
        return st["ms"], st
    if algo == "sssp":
        _, st = dag.sssp(plan, kw["src"], kw["w"], variant=variant, delta=delta)
        return st["ms"], st
    if algo == "ppr_batched":
        _, _, st = dag.ppr_batched(plan, kw["V"], variant=variant, delta=delta, tol=kw.get("tol", 1e-6))
        return st["ms"], st
    if algo == "sssp_batched":
        _, _, st = dag.sssp_batched(plan, kw["srcs"], kw["w"], variant=variant, delta=delta)
        return st["ms"], st
    raise ValueError(algo)


def tune(plan: dag.Plan, algo: str, candidates=None, worker_fractions=None, trials: int = 2,
         cache: str | None = DEFAULT_CACHE, **kw) -> dict:
    """Fastest (variant, delta, workers) for `algo` on this plan's graph.

    algo: "pagerank" (kw: tol, teleport, ...), "sssp" (kw: src, w), "ppr_batched"
    (kw: V), "sssp_batched" (kw: srcs, w). Returns a dict with the choice and the
    measured candidates; leaves the plan's worker cap at the chosen value.
    """
    batched = algo.endswith("batched")
    cands = candidates or (BATCH_CANDIDATES if batched else SINGLE_CANDIDATES)
    fracs = worker_fractions or WORKER_FRACTIONS
    B = int(kw["V"].shape[1]) if algo == "ppr_batched" else (int(kw["srcs"].numel()) if algo == "sssp_batched" else 1)
    key = f"{fingerprint(plan)}|{algo}|B{B}"
    if cache:
        hit = _load(cache).get(key)
        if hit:
            plan.set_worker_cap(hit["workers"])
            return hit
    plan.set_worker_cap(0)
    full = plan.workers("async", 0)
    results = []
    for frac in fracs:
        cap = max(1, int(full * frac))
        plan.set_worker_cap(0 if frac >= 1.0 else cap)
        for variant, delta in cands:
            times, sweeps = [], []
            try:
                for _ in range(trials):
                    ms, st = _run(plan, algo, variant, delta, kw)
                    times.append(ms)
                    sweeps.append(st.get("iters", st.get("sweeps")))
            except dag.DagError as e:  # e.g. a delta whose buffer cannot be resident
                results.append(dict(variant=variant, delta=delta, workers=0 if frac >= 1.0 else cap,
                                    error=str(e)))
                continue
            results.append(dict(variant=variant, delta=delta, workers=0 if frac >= 1.0 else cap,
                                ms=float(np.median(times)), sweeps=sweeps))
    ok = [r for r in results if "ms" in r]
    best = min(ok, key=lambda r: r["ms"])
    choice = dict(variant=best["variant"], delta=best["delta"], workers=best["workers"], ms=best["ms"],
                  candidates=results)
    plan.set_worker_cap(best["workers"])
    if cache:
        _store(cache, key, choice)
    torch.cuda.synchronize()
    return choice
