"""Benchmark: delayed-asynchronous PageRank + Bellman-Ford on RMAT scale 22.

One step = one PageRank solve (d = 0.85, tol 1e-6) plus eight Bellman-Ford
solves (fixed sources, one-byte weights in [1, 255]) on the RMAT scale-22 graph
(a=.57 b=.19 c=.19, edge factor 16, seed 2), all in the persistent CUDA
kernels behind the C ABI, each with the delayed method's buffer size delta
picked by the autotuner among {0, 32, 256, 4096} (delta = 0 is the
asynchronous end of the method, Sec. III-B). The metric is GTEPS counted per
finished solve: (solves * m) / time. With inputs resident in HBM the timed
region holds K steps between CUDA events; `e2e` repeats the step through the
public API from pinned host buffers (graph upload, plan, solves, result
download). The CSR (about 285 MB) and weights are larger than L2, so no flush
is needed between steps.

--impl reference times the CPU oracle's OpenMP form of the same method (the
paper's CPU scheme) on the host cores, on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PageRank/SSSP time-to-converge & GTEPS at tol 1e-6; batched & adjoint vs plain"
SCALE, EF, SEED = 22, 16, 2
N_SOURCES = 8
PR_DELTA, SSSP_DELTA = 32, 32  # fixed-delta runs of the variant table and the CPU oracle
DELTAS = (0, 32, 256, 4096)
WORKLOAD = (f"rmat{SCALE}: pagerank d=0.85 tol=1e-6 + sssp x{N_SOURCES} sources, "
            f"delayed method, delta picked per algorithm over {list(DELTAS)} "
            f"(delta 0 also with own-block or all L1 reads, and for sssp the tile frontier on CTA tiles, warp runs "
            f"or CTA-ordered warp tiles) "
            f"and over warp-worker sweeps (sync, delta 16 / 256, async with three warp tile shapes) "
            f"and ordered warp sweeps (async, two warp tile shapes)")


HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (the roofline's frac uses the measured copy peak)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def replica_aggregate(ms_local, world, edges_per_rank, device):
    """Whole-job result of N independent replicas: the slowest rank's time
    (max over ranks) and every rank's solved edges over it, in GTEPS. With one
    rank there is nothing to exchange."""
    if world > 1:
        import torch
        import torch.distributed as dist

        tt = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_local = float(tt.item())
        dist.barrier()
    return ms_local, world * edges_per_rank / (ms_local * 1e-3) / 1e9


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str | None = None):
        self.index = index
        self.proc = None
        # the samples go to --clocks-csv (rank-suffixed) when given, else to a temporary file
        if path:
            root, ext = os.path.splitext(path)
            self.path = f"{root}_rank{index}{ext or '.csv'}"
        else:
            import tempfile

            self.path = os.path.join(tempfile.gettempdir(), f"dag_bench_clocks_{os.getpid()}_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def build_inputs():
    from paper_2110_01409_gb300 import inputs as I

    t0 = time.time()
    g = I.rmat(SCALE, EF, 0.57, 0.19, 0.19, seed=SEED)
    w = I.weights_u32(g, SEED)
    srcs = I.sources(g, N_SOURCES, seed=SEED)
    return g, w, srcs, time.time() - t0


def _cand(c):
    v = "sync" if c["variant"] == "sync" else str(c["delta"])
    tile = f"x{c['warp_tile']}" if c["reads"].startswith(("warp", "ordered")) else ""
    return v + ("" if c["reads"] == "refresh" else "+" + c["reads"]) + tile


def algorithmic_bytes(n, m, kind, edges=None):
    """Compulsory bytes of one sweep (gathers of the state vector count as L2
    hits: the 4n-byte vector fits in L2): rowptr 4(n+1), colidx 4m, own old
    value 4n + new value 4n, plus per-vertex out-degree 4n (PageRank) or the
    per-edge weight (Bellman-Ford: 4m as uint32, m as uint8). With `edges`
    (a frontier launch: the edges it ran over all its sweeps) the result is
    per launch: the per-edge terms count those edges, the per-vertex ones are
    left to the caller's sweep count."""
    per_vertex = 4 * (n + 1) + 8 * n + (4 * n if kind == "pr" else 0)
    per_edge = 4 + {"pr": 0, "bf": 4, "bf8": 1}[kind]
    if edges is None:
        return per_vertex + per_edge * m
    return per_edge * edges, per_vertex


def run_gpu(args):
    import torch

    from paper_2110_01409_gb300 import build as B
    from paper_2110_01409_gb300 import dag

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    g, w, srcs, gen_s = build_inputs()
    n, m = g.n, g.m
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rowptr = torch.from_numpy(g.rowptr).to(dev)
    colidx = torch.from_numpy(g.colidx).to(dev)
    w_d = torch.from_numpy(w.view(np.int32)).to(dev)      # uint32 weights (variant table, reference runs)
    w8_d = torch.from_numpy(w.astype(np.uint8)).to(dev)   # the same weights, one byte each (w <= 255)
    plan = dag.Plan(rowptr, colidx)
    rank_out = torch.empty(n, dtype=torch.float32, device=dev)
    dist_out = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(N_SOURCES)]

    # ---- delta per algorithm: the autotuner over the delayed method's delta (0 = async end) ----
    from paper_2110_01409_gb300 import autotune

    # CTA-tile sweeps over delta, plus warp-worker sweeps (three warp tile shapes for the async end)
    warp_cands = [("sync", 0, "warp"), ("delayed", 16, "warp"), ("delayed", 256, "warp+cached")] + \
        [("delayed", 0, "warp+cached", ipt) for ipt in (5, 7, 11)] + \
        [("delayed", 0, "ordered+cached", ipt) for ipt in (7, 11)]
    cands = [("delayed", dl) for dl in DELTAS] + [("delayed", 0, "own_l1"), ("delayed", 0, "cached")] + warp_cands
    cands_bf = cands + [("delayed", 0, "frontier"), ("delayed", 0, "own_l1+frontier"), ("delayed", 0, "cached+frontier"),
                        ("delayed", 0, "warp+frontier"), ("delayed", 0, "warp+cached+frontier"),
                        ("delayed", 0, "ordered+frontier"), ("delayed", 0, "ordered+cached+frontier")]
    tune_pr = autotune.tune(plan, "pagerank", candidates=cands, worker_fractions=[1.0], trials=2, cache=None)
    tune_bf = autotune.tune(plan, "sssp", candidates=cands_bf, worker_fractions=[1.0], trials=2, cache=None,
                            src=int(srcs[0]), w=w8_d)
    plan.set_worker_cap(0)
    pr_dl, bf_dl = tune_pr["delta"], tune_bf["delta"]
    pr_rd, bf_rd = tune_pr["reads"], tune_bf["reads"]
    pr_var, bf_var = tune_pr["variant"], tune_bf["variant"]
    pr_tile, bf_tile = tune_pr["warp_tile"], tune_bf["warp_tile"]

    def pagerank_solve(**kw):  # the tuned choice (its warp tile is a host-side plan setting)
        plan.set_warp_tile(pr_tile)
        return dag.pagerank(plan, 0.85, 1e-6, pr_var, pr_dl, 1000, out=rank_out, reads=pr_rd, **kw)

    def sssp_solve(s, k, **kw):
        plan.set_warp_tile(bf_tile)
        return dag.sssp(plan, int(s), w8_d, bf_var, bf_dl, n + 1, out=dist_out[k], reads=bf_rd, **kw)

    # ---- warm-up with statuses (also records per-solve sweeps) ----
    pr_iters, bf_iters, bf_edges = [], [], []
    for _ in range(args.warmup):
        _, st = pagerank_solve()
        assert st["converged"], st
        pr_iters.append(st["iters"])
        its = []
        for k, s in enumerate(srcs):
            _, st = sssp_solve(s, k)
            assert st["converged"], st
            its.append(st["iters"])
            bf_edges.append(st["edges_processed"])
        bf_iters.append(its)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device events, per-launch events for the roofline ----
    K = args.steps
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    pr_ev = [(ev(), ev()) for _ in range(K)]
    bf_ev = [[(ev(), ev()) for _ in range(N_SOURCES)] for _ in range(K)]
    t_start, t_end = ev(), ev()
    status = torch.zeros((K, 1 + N_SOURCES, 3), dtype=torch.int32, device=dev)  # each timed solve's status
    clocks = Clocks(local, args.clocks_csv)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start.record(stream)
    for k in range(K):
        pr_ev[k][0].record(stream)
        pagerank_solve(stats=False)
        pr_ev[k][1].record(stream)
        plan.last_status_to(status[k, 0])
        for j, s in enumerate(srcs):
            bf_ev[k][j][0].record(stream)
            sssp_solve(s, j, stats=False)
            bf_ev[k][j][1].record(stream)
            plan.last_status_to(status[k, 1 + j])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    solves = 1 + N_SOURCES
    ms_total, value = replica_aggregate(ms_total, world, solves * m * K, dev)
    ms_step = ms_total / K

    # every timed solve converged without error (read on the device, checked after the region)
    st_all = status.cpu()
    assert bool((st_all[..., 0] == 0).all()) and bool((st_all[..., 1] == 1).all()), st_all
    _, st_pr = pagerank_solve()
    assert st_pr["converged"]
    pr_ms = statistics.mean(a.elapsed_time(b) for a, b in pr_ev)
    bf_ms = statistics.mean(a.elapsed_time(b) for row in bf_ev for a, b in row)
    pr_sweeps = statistics.mean(pr_iters + [st_pr["iters"]])
    bf_sweeps = statistics.mean(x for row in bf_iters for x in row)
    pr_bytes = algorithmic_bytes(n, m, "pr") * pr_sweeps
    bf_edges_mean = statistics.mean(bf_edges)  # m per sweep, or the frontier's edges per launch
    e_bytes, v_bytes = algorithmic_bytes(n, m, "bf8", edges=bf_edges_mean)
    bf_bytes = e_bytes + v_bytes * bf_sweeps
    peak, peak_kind = _peaks()
    # dominant kernel by total time in the step
    if bf_ms * N_SOURCES >= pr_ms:
        dom, dom_bytes, dom_ms, dom_sweeps = kernel_name("BF8", bf_var, bf_dl, bf_rd, bf_tile), bf_bytes, bf_ms, \
            bf_sweeps
    else:
        dom, dom_bytes, dom_ms, dom_sweeps = kernel_name("PR", pr_var, pr_dl, pr_rd, pr_tile), pr_bytes, pr_ms, \
            pr_sweeps
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = _recorded_traffic(dom, dom_sweeps, bf_edges_mean if "frontier" in dom else None)

    # ---- the delayed variant's own fraction: the fastest delta > 0 candidate of each algorithm ----
    def delayed_roof(tuned, kind, mode):
        best = min((c for c in tuned["candidates"] if "ms" in c and c["variant"] == "delayed" and c["delta"] > 0),
                   key=lambda c: c["ms"], default=None)
        if best is None:
            return None
        sweeps = statistics.mean(best["sweeps"])
        gbs = algorithmic_bytes(n, m, kind) * sweeps / (best["ms"] * 1e-3) / 1e9
        kern = kernel_name(mode, "delayed", best["delta"], best["reads"], best["warp_tile"])
        return {"kernel": kern, "delta": best["delta"], "reads": best["reads"], "ms": round(best["ms"], 3),
                "sweeps": sweeps, "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                "traffic": _recorded_traffic(kern, sweeps)}

    delayed_roofline = {"pagerank": delayed_roof(tune_pr, "pr", "PR"), "sssp": delayed_roof(tune_bf, "bf8", "BF8")}

    # ---- the sweep's real ceiling: one streamed gather pass over the same colidx (dag_probe_gather) ----
    coherent = gathers_coherent(bf_var, bf_dl, bf_rd)
    probe_ms = dag.probe_gather(plan, rank_out, coherent=coherent, repeats=5)
    # the launch against the probe's time for the edges it ran (sweeps * m, or the frontier's count)
    bf_sweep_ms = bf_ms / bf_sweeps
    gather_floor = {"probe_ms_per_pass": round(probe_ms, 4), "loads": "relaxed (L2)" if coherent else "ordinary",
                    "sweep_ms": round(bf_sweep_ms, 4), "edges_per_launch_over_m": round(bf_edges_mean / m, 3),
                    "frac": round(probe_ms * (bf_edges_mean / m) / bf_ms, 3),
                    "kernel": kernel_name("BF8", bf_var, bf_dl, bf_rd, bf_tile)}

    # ---- e2e through the public API from pinned host buffers ----
    # e2e builds a plan per step and runs the device step's own choices; a frontier choice builds its
    # out-edge maps (a counting sort of the in-CSR by source) inside the first solve of every step
    bf_choice_e2e = (bf_var, bf_dl, bf_rd, bf_tile)
    e2e = run_e2e(args, g, w, srcs, dev, dag, torch, (pr_var, pr_dl, pr_rd, pr_tile), bf_choice_e2e) \
        if args.e2e else None
    if e2e is not None:
        e2e["sssp_reads"] = bf_choice_e2e[2]
        e2e["sssp_warp_tile_items"] = 32 * bf_choice_e2e[3] if dag.uses_warp_tile(bf_choice_e2e[2]) else None

    detail = {}
    if args.extras and rank == 0:
        detail["variants"] = run_detail(g, w, srcs, plan, w_d, dag, torch, args)
        detail["adjoint"] = run_adjoint(g, plan, dag, torch)
        detail["batched"] = run_batched(dag, torch)
        detail["access"] = run_access(g, plan, dag, torch)
        detail["config3"] = run_config3(dag, torch)

    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GTEPS",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32/u32",
        "data": "synthetic (seeded RMAT stand-in for the GAP Kron graph)",
        "config": {"workload": WORKLOAD, "weights": "uint8 per edge (values in [1, 255])",
                   "variant": {"pagerank": pr_var, "sssp": bf_var},
                   "delta": {"pagerank": pr_dl, "sssp": bf_dl},
                   "reads": {"pagerank": pr_rd, "sssp": bf_rd},
                   "warp_tile_items": {"pagerank": 32 * pr_tile if pr_rd.startswith(("warp", "ordered")) else None,
                                       "sssp": 32 * bf_tile if bf_rd.startswith(("warp", "ordered")) else None},
                   "autotune_ms": {"pagerank": {_cand(c): round(c["ms"], 3) for c in tune_pr["candidates"]
                                                if "ms" in c},
                                   "sssp": {_cand(c): round(c["ms"], 3) for c in tune_bf["candidates"]
                                            if "ms" in c}},
                   "n": n, "m": m, "sources": [int(s) for s in srcs], "workers": st_pr["workers"],
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (CSR + one-byte weights 0.34 GB)",
                   "graph_gen_s": round(gen_s, 2)},
        "per_solve": {"pagerank_ms": round(pr_ms, 3), "pagerank_sweeps": pr_sweeps,
                      "sssp_ms": round(bf_ms, 3), "sssp_sweeps": bf_sweeps,
                      "gteps_work_rate": round(((pr_sweeps + N_SOURCES * bf_sweeps) * m) / (ms_step * 1e-3) / 1e9, 3)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "frac_of_nominal": round(achieved / HBM_NOMINAL_GBS, 4),
                     "bytes_per_launch": int(dom_bytes), "traffic": traffic},
        "gather_floor": gather_floor,
        "delayed_roofline": delayed_roofline,
        "clocks": clk,
        "gpu_launches": 2 * K * solves,  # each solve's sweep kernel and its status copy
        "e2e": e2e,
    }
    if rank == 0 and args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, w, srcs)
    if detail:
        out["detail"] = detail
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def kernel_name(mode, variant, delta, reads, warp_tile=7):
    """The sweep kernel a solve runs (for the roofline's kernel and the ncu launch list)."""
    var = "ASYNC" if variant == "async" or (variant == "delayed" and delta == 0) else variant.upper()
    if reads.startswith(("warp", "ordered")) and "frontier" in reads:
        return f"sweep_warp_frontier_kernel<{mode},{warp_tile}{',ordered' if reads.startswith('ordered') else ''}>"
    if reads.startswith("warp"):
        return f"sweep_warp_kernel<{mode},{var},{warp_tile}>"
    if reads.startswith("ordered"):
        return f"sweep_ordered_kernel<{mode},{warp_tile}>"
    if var == "ASYNC":
        return f"sweep_tma_kernel<{mode}{',frontier' if 'frontier' in reads else ''}>"
    return f"sweep_kernel<{mode},{var}{',frontier' if 'frontier' in reads else ''}>"


def gathers_coherent(variant, delta, reads):
    """True when the solve gathers with gpu-scope loads served by L2 (the async form's default)."""
    asynch = variant == "async" or (variant == "delayed" and delta == 0)
    return ("coherent" in reads) or (asynch and "cached" not in reads)  # own_l1: other blocks through L2


SWEEP_SOURCES = ("sweep.cu", "sweep_tma.cu", "sweep_warp.cu", "sweep_warp_frontier.cu", "sweep_warp.cuh",
                 "sweep_common.cuh", "dag_internal.cuh")


def sweep_source_hash():
    """sha256 of the sweep kernel's sources: a recorded ncu traffic figure is
    used only while it still describes the kernel that runs."""
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2110_01409_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _recorded_traffic(kernel, sweeps, edges=None):
    """DRAM bytes per launch (read + write) from profiles/sweep_traffic.txt, a
    summary of an ncu capture of the same kernel on the same workload, scaled
    by the launch's sweeps (a frontier launch: by the edges it ran); None when
    the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "sweep_traffic.txt")
    try:
        rec = {}
        with open(path) as f:
            for line in f:
                if line.strip() and not line.startswith("#") and ":" in line:
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        if rec.get("sweep_source_sha256") != sweep_source_hash():
            return None
        if "frontier" in kernel:
            return int(float(rec[f"{kernel} rmat{SCALE} dram_bytes_per_edge_run"]) * edges)
        per_sweep = float(rec[f"{kernel} rmat{SCALE} dram_bytes_per_sweep"])
        return int(per_sweep * sweeps)
    except Exception:
        return None


def run_e2e(args, g, w, srcs, dev, dag, torch, pr_choice, bf_choice):
    """Same step through the public API from pinned host memory, copies inside the timed region."""
    rp_h = torch.from_numpy(g.rowptr).pin_memory()
    ci_h = torch.from_numpy(g.colidx).pin_memory()
    w_h = torch.from_numpy(w.astype(np.uint8)).pin_memory()
    res_pr = torch.empty(g.n, dtype=torch.float32).pin_memory()
    res_bf = torch.empty((N_SOURCES, g.n), dtype=torch.int32).pin_memory()
    h2d = rp_h.numel() * 4 + ci_h.numel() * 4 + w_h.numel() * 1
    d2h = res_pr.numel() * 4 + res_bf.numel() * 4
    K = max(1, min(args.steps, 3))

    side = torch.cuda.Stream()  # copies that overlap the solves: the weights in, the results out

    def step():
        main = torch.cuda.current_stream()
        rp = rp_h.to(dev, non_blocking=True)
        ci = ci_h.to(dev, non_blocking=True)
        with torch.cuda.stream(side):  # the weights arrive while the plan is built and PageRank runs
            wd = w_h.to(dev, non_blocking=True)
        w_ready = side.record_event()
        wd.record_stream(main)
        plan = dag.Plan(rp, ci)
        plan.set_warp_tile(pr_choice[3])
        r, _ = dag.pagerank(plan, 0.85, 1e-6, pr_choice[0], pr_choice[1], 1000, stats=False, reads=pr_choice[2])
        side.wait_event(main.record_event())
        with torch.cuda.stream(side):
            res_pr.copy_(r, non_blocking=True)
        r.record_stream(side)
        main.wait_event(w_ready)
        plan.set_warp_tile(bf_choice[3])
        for j, s in enumerate(srcs):
            d, _ = dag.sssp(plan, int(s), wd, bf_choice[0], bf_choice[1], g.n + 1, stats=False, reads=bf_choice[2])
            side.wait_event(main.record_event())  # this result goes out while the next source runs
            with torch.cuda.stream(side):
                res_bf[j].copy_(d, non_blocking=True)
            d.record_stream(side)
        torch.cuda.synchronize()
        plan.close()

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        step()
    t = (time.perf_counter() - t0) / K
    return {"value": round((1 + N_SOURCES) * g.m / t / 1e9, 3), "unit": "GTEPS", "ms_per_step": round(t * 1e3, 3),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def _variant_rows(dag, torch, plan, g, src, w_d, variants, trials=3):
    """Median time and sweeps of each (name, variant, delta, reads[, warp tile]) row for PageRank
    and Bellman-Ford; frontier rows are Bellman-Ford only. Also the edges the SSSP solves ran.
    Warp-tile rows run 32 x 7 items unless the row names another shape."""
    res = {}
    for row_spec in variants:
        name, var, dl, rd = row_spec[:4]
        plan.set_warp_tile(row_spec[4] if len(row_spec) > 4 else 7)
        pr_it, pr_ms, bf_it, bf_ms = [], [], [], []
        for _ in range(trials):
            if "frontier" not in rd:
                _, st = dag.pagerank(plan, 0.85, 1e-6, var, dl, 1000, reads=rd)
                assert st["converged"], (name, st)
                pr_it.append(st["iters"])
                pr_ms.append(st["ms"])
            _, st = dag.sssp(plan, src, w_d, var, dl, g.n + 1, reads=rd)
            assert st["converged"], (name, st)
            bf_it.append(st["iters"])
            bf_ms.append(st["ms"])
        row = {"sssp_sweeps": bf_it, "sssp_ms_median": round(statistics.median(bf_ms), 3),
               "sssp_edges_per_m": round(st["edges_processed"] / max(g.m, 1), 2)}
        if pr_ms:
            row.update({"pr_sweeps": pr_it, "pr_ms_median": round(statistics.median(pr_ms), 3)})
        res[name] = row
    torch.cuda.synchronize()
    return res


VARIANT_ROWS = [("sync", "sync", 0, "refresh"), ("async", "async", 0, "refresh"),
                ("async_own_l1", "async", 0, "own_l1"), ("sync_frontier", "sync", 0, "frontier"),
                ("async_frontier", "async", 0, "frontier"), ("async_own_l1_frontier", "async", 0, "own_l1+frontier"),
                ("async_cached", "async", 0, "cached"), ("async_cached_frontier", "async", 0, "cached+frontier"),
                ("warp_async_frontier", "async", 0, "warp+frontier"),
                ("warp_async_cached_frontier", "async", 0, "warp+cached+frontier"),
                ("ordered_cached_frontier", "async", 0, "ordered+cached+frontier"),
                ("delayed32", "delayed", 32, "refresh"), ("delayed256", "delayed", 256, "refresh"),
                ("delayed4096", "delayed", 4096, "refresh"), ("delayed4096_local", "delayed", 4096, "local"),
                ("warp_sync", "sync", 0, "warp"), ("warp_async_cached", "async", 0, "warp+cached"),
                ("warp_delayed16", "delayed", 16, "warp"), ("warp_delayed256_cached", "delayed", 256, "warp+cached"),
                ("ordered_cached", "async", 0, "ordered+cached", 11)]


def run_detail(g, w, srcs, plan, w_d, dag, torch, args):
    """Per-variant sweeps and times (3 trials) on the benchmark graph (Bellman-Ford with
    four-byte weights); the paper's variants table."""
    return _variant_rows(dag, torch, plan, g, int(srcs[0]), w_d, VARIANT_ROWS)


def run_config3(dag, torch):
    """The clustered and uniform graphs at full size: banded n = 2^24 (15 edges within
    +-1024 + 1 uniform) and ER n = 2^23 (16 per vertex), seed 3; PageRank and
    Bellman-Ford (one-byte weights) in every variant; 3 trials each."""
    import paper_2110_01409_gb300.inputs as I

    out = {}
    variants = VARIANT_ROWS
    for gname, make in (("banded24", lambda: I.banded(1 << 24, 15, 1024, 1, seed=3)),
                        ("er23", lambda: I.erdos_renyi(1 << 23, 16, seed=3))):
        t0 = time.time()
        g = make()
        gen_s = time.time() - t0
        pl = dag.Plan.from_graph(g, "cuda")
        w8 = torch.from_numpy(I.weights_u32(g, 3).astype(np.uint8)).cuda()
        src = int(I.sources(g, 1, seed=3)[0])
        tab = {"n": g.n, "m": g.m, "graph_gen_s": round(gen_s, 1),
               "locality_P32": round(dag.locality(dag.access_matrix(pl, 32))["diag_share"], 4)}
        tab.update(_variant_rows(dag, torch, pl, g, src, w8, variants))
        pl.close()
        del w8
        out[gname] = tab
    torch.cuda.synchronize()
    return out


def run_access(g, plan, dag, torch):
    """Fig. 5: reads by each worker of every worker's block, for the benchmark's RMAT
    graph and a banded graph of the same size (local clustering), at 32 workers
    (the paper's thread count) and at the sweep's CTA count."""
    import paper_2110_01409_gb300.inputs as I

    out = {}
    banded = I.banded(g.n, 15, 1024, 1, seed=SEED)
    bplan = dag.Plan.from_graph(banded, "cuda")
    for name, pl in (("rmat", plan), ("banded", bplan)):
        for P in (32, pl.workers("async", 0)):
            st = dag.locality(dag.access_matrix(pl, P))
            out[f"{name}_P{P}"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()}
    # global vs local reads (Sec. III-C) where a worker reads mostly its own block
    wb = torch.from_numpy(I.weights_u32(banded, SEED).astype(np.uint8)).cuda()
    src = int(I.sources(banded, 1, seed=SEED)[0])
    tab = _variant_rows(dag, torch, bplan, banded, src, wb, VARIANT_ROWS)
    out["banded_variants"] = tab
    bplan.close()
    torch.cuda.synchronize()
    return out


def cpu_tune(g, w, src, cores):
    """Best delta per algorithm for the CPU oracle's OpenMP form (one trial each)."""
    import oracle

    best_pr = min(DELTAS, key=lambda dl: oracle.pagerank_threads(g, oracle.DELAYED, tol=1e-6, threads=cores,
                                                                 delta=dl)[2])
    best_bf = min(DELTAS, key=lambda dl: oracle.sssp_threads(g, w, src, oracle.DELAYED, threads=cores, delta=dl)[2])
    return best_pr, best_bf


def cpu_step(g, w, srcs, cores, pr_dl, bf_dl):
    """One step on the CPU oracle's OpenMP form (the paper's thread scheme):
    1 PageRank + the 8 Bellman-Ford solves. Returns seconds, sweeps, converged."""
    import oracle

    _, it_pr, s_pr, ok = oracle.pagerank_threads(g, oracle.DELAYED, tol=1e-6, threads=cores, delta=pr_dl)
    secs, sweeps = s_pr, [it_pr]
    for s in srcs:
        _, it, sec, ok2 = oracle.sssp_threads(g, w, int(s), oracle.DELAYED, threads=cores, delta=bf_dl)
        secs += sec
        sweeps.append(it)
        ok = ok and ok2
    return secs, sweeps, ok


def cpu_baseline(g, w, srcs):
    """The oracle's OpenMP form on all host cores, on the whole step (bounded: a few seconds)."""
    cores = os.cpu_count() or 1
    pr_dl, bf_dl = cpu_tune(g, w, int(srcs[0]), cores)
    secs, sweeps, ok = cpu_step(g, w, srcs, cores, pr_dl, bf_dl)
    # one thread, one PageRank solve (the same form; bounded to a couple of seconds)
    _, it1, s1, _ = oracle_pr_threads(g, pr_dl, 1)
    return {"value": round((1 + N_SOURCES) * g.m / secs / 1e9, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": f"one full step (1 pagerank + {N_SOURCES} sssp, delta {pr_dl}/{bf_dl} picked over "
                      f"{list(DELTAS)}, sweeps {sweeps}) in {secs:.2f} s", "converged": bool(ok),
            "single_thread": {"value": round(g.m / s1 / 1e9, 4), "unit": "GTEPS",
                              "sample": f"one pagerank solve on 1 thread, delta {pr_dl}, {it1} sweeps, {s1:.2f} s"}}


def oracle_pr_threads(g, delta, threads):
    import oracle

    return oracle.pagerank_threads(g, oracle.DELAYED, tol=1e-6, threads=threads, delta=delta)


def run_reference(args):
    """Reference arm: the CPU oracle's paper-scheme form, timed on the host cores."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    g, w, srcs, _ = build_inputs()
    cores = os.cpu_count() or 1
    pr_dl, bf_dl = cpu_tune(g, w, int(srcs[0]), cores)
    for _ in range(args.warmup):
        cpu_step(g, w, srcs, cores, pr_dl, bf_dl)
    t = 0.0
    for _ in range(args.steps):
        secs, _, _ = cpu_step(g, w, srcs, cores, pr_dl, bf_dl)
        t += secs
    value = (1 + N_SOURCES) * g.m * args.steps / t / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/u32",
           "data": "synthetic (seeded RMAT stand-in for the GAP Kron graph)",
           "config": {"workload": WORKLOAD, "delta": {"pagerank": pr_dl, "sssp": bf_dl}, "n": g.n, "m": g.m},
           "cpu_baseline": {"value": round(value, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                            "sample": "each step: the full step (1 pagerank + 8 sssp) on the oracle's OpenMP form"},
           "e2e": {"value": round(value, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched(dag, torch):
    """Batched form (RMAT scale 20, seed 4): 256 PPR columns + 64 SSSP sources, one
    persistent launch each, against the plain single-vector sweep on the same graph."""
    from paper_2110_01409_gb300 import autotune
    from paper_2110_01409_gb300 import inputs as I

    g = I.rmat(20, 16, 0.57, 0.19, 0.19, seed=4)
    plan = dag.Plan.from_graph(g, "cuda")
    sets = I.ppr_seed_sets(g.n, 256, seed=4)
    V = torch.from_numpy(I.teleport_matrix(g.n, sets)).cuda()
    w = torch.from_numpy(I.weights_u32(g, 4).astype(np.uint8)).cuda()  # one-byte weights (values in [1, 255])
    srcs = torch.from_numpy(I.sources(g, 64, seed=4).view(np.int32)).cuda()
    tuned_ppr = autotune.tune(plan, "ppr_batched", cache=None, trials=1, V=V)
    R, it, st = dag.ppr_batched(plan, V, 0.85, 1e-6, tuned_ppr["variant"], tuned_ppr["delta"])
    tuned_bf = autotune.tune(plan, "sssp_batched", cache=None, trials=1, srcs=srcs, w=w)
    D, it2, st2 = dag.sssp_batched(plan, srcs, w, tuned_bf["variant"], tuned_bf["delta"])
    plan.set_worker_cap(0)
    # plain single-vector solves of a few columns with the same choice, for the per-column comparison
    one_ppr, one_bf = [], []
    Vc = V[:, :8].t().contiguous()
    for c in range(8):
        _, s1 = dag.pagerank(plan, 0.85, 1e-6, "async", 0, teleport=Vc[c].contiguous())
        one_ppr.append(s1["ms"])
        _, s2 = dag.sssp(plan, int(srcs[c]), w, "async", 0, reads="own_l1+frontier")
        one_bf.append(s2["ms"])
    m, n = g.m, g.n
    peak, peak_kind = _peaks()

    def roof(nbytes, ms):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(gbs / peak, 4), "bytes_per_launch": int(nbytes)}

    # algorithmic bytes: the CSR once per sweep, per active column its own rows (12n PPR: teleport, old,
    # new; 8n SSSP: old, new) and its gathers (4m: X[n][B] is far larger than L2); weights once per sweep
    ppr_bytes = st["sweeps"] * (4 * (n + 1) + 4 * m) + st["column_sweeps"] * (12 * n + 4 * m)
    bf_bytes = st2["sweeps"] * (4 * (n + 1) + 5 * m) + st2["column_sweeps"] * (8 * n + 4 * m)
    return {"graph": {"n": g.n, "m": m, "seed": 4},
            "roofline": {"ppr": roof(ppr_bytes, st["ms"]), "sssp": roof(bf_bytes, st2["ms"])},
            "cuda_graph": {"ppr": st["graph"], "sssp": st2["graph"]},
            "ppr": {"B": 256, "choice": {k: tuned_ppr[k] for k in ("variant", "delta", "workers")},
                    "ms": round(st["ms"], 3), "sweeps": st["sweeps"], "column_sweeps": st["column_sweeps"],
                    "gteps_solve_rate": round(256 * m / (st["ms"] * 1e-3) / 1e9, 2),
                    "single_vector_ms_per_column": round(float(np.median(one_ppr)), 3),
                    "speedup_vs_single": round(256 * float(np.median(one_ppr)) / st["ms"], 2),
                    "converged": st["converged"]},
            "sssp": {"B": 64, "choice": {k: tuned_bf[k] for k in ("variant", "delta", "workers")},
                     "ms": round(st2["ms"], 3), "sweeps": st2["sweeps"], "column_sweeps": st2["column_sweeps"],
                     "gteps_solve_rate": round(64 * m / (st2["ms"] * 1e-3) / 1e9, 2),
                     "single_vector_ms_per_source": round(float(np.median(one_bf)), 3),
                     "speedup_vs_single": round(64 * float(np.median(one_bf)) / st2["ms"], 2),
                     "converged": st2["converged"]}}


def run_adjoint(g, plan, dag, torch):
    """Adjoint form (RMAT scale 22, FP32 weights in (0,1], 4096 targets, w_i ~ N(0,1)):
    forward weighted PageRank and its backward pass, beside the plain sweep. The headline pair is
    the asynchronous form on warp workers with cached reads (forward and adjoint alike); the
    synchronous warp form, the ordered warp sweep and the CTA-tile asynchronous form are reported
    beside it."""
    from paper_2110_01409_gb300 import inputs as I

    w = torch.from_numpy(I.weights_f32(g, SEED)).cuda()
    targets, wt = I.adjoint_targets(g.n, 4096, seed=5)
    c = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    c[torch.from_numpy(targets).cuda()] = torch.from_numpy(wt.astype(np.float32)).cuda()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    forms = {}
    plan.set_warp_tile(7)
    for name, variant, reads in (("warp_async_cached", "async", "warp+cached"), ("warp_sync", "sync", "warp"),
                                 ("ordered_cached", "async", "ordered+cached"), ("cta_async", "async", "refresh")):
        model = dag.WeightedPageRank(plan, d=0.85, tol=1e-6, variant=variant, delta=0, reads=reads)
        for rep in range(2):
            e0, e1, e2 = ev(), ev(), ev()
            e0.record()
            r, val, s, st_f = model.forward(w)
            e1.record()
            gw, gt, _, st_b = model.backward(val, s, r, c)
            e2.record()
            torch.cuda.synchronize()
            # forward_ms includes the weight normalisation (its out-CSR order is built on the plan's first
            # call, in rep 0); backward_ms the gather of the weights into out-edge order; adjoint_solve_ms
            # is the adjoint solve with the edge gradients, against the forward solve alone
            forms[name] = {"variant": variant, "reads": reads, "forward_ms": round(e0.elapsed_time(e1), 3),
                           "forward_solve_ms": round(st_f["ms"], 3), "forward_sweeps": st_f["iters"],
                           "backward_ms": round(e1.elapsed_time(e2), 3), "adjoint_sweeps": st_b["iters"],
                           "adjoint_solve_ms": round(st_b["ms"], 3), "targets": 4096,
                           "backward_over_forward_solve": round(st_b["ms"] / st_f["ms"], 3),
                           "converged": bool(st_f["converged"] and st_b["converged"])}
        model.out_plan.close()
    out = dict(forms["warp_async_cached"])
    out["other_forms"] = {k: v for k, v in forms.items() if k != "warp_async_cached"}
    return out


def run_gpu_rowshard(args):
    """--shard rows: the same step (1 PageRank + 8 Bellman-Ford, synchronous) with the rows of one
    graph split over the ranks (rowshard.py): every sweep each rank computes its Sec. III-A row
    range on its GPU, then an all-gather of the ranges and an all-reduce of the FP64 sums. Total
    work is fixed as ranks are added ("scaling": "strong")."""
    import torch

    from paper_2110_01409_gb300 import build as B
    from paper_2110_01409_gb300 import dag
    from paper_2110_01409_gb300 import rowshard as RS

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    g, w, srcs, gen_s = build_inputs()
    n, m = g.n, g.m
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    plan = dag.Plan(torch.from_numpy(g.rowptr).to(dev), torch.from_numpy(g.colidx).to(dev))
    w8 = torch.from_numpy(w.astype(np.uint8)).to(dev)

    def step():
        r, it_pr, ok = RS.pagerank_row_sharded(dag, plan, rank, world)
        its = [it_pr]
        for s in srcs:
            _, it, ok2 = RS.sssp_row_sharded(dag, plan, int(s), w8, rank, world)
            ok = ok and ok2
            its.append(it)
        return its, ok

    for _ in range(args.warmup):
        its, ok = step()
        assert ok, its
    K = args.steps
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local, args.clocks_csv)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    sweeps = []
    for _ in range(K):
        its, ok = step()
        assert ok, its
        sweeps.append(its)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_local = t0.elapsed_time(t1)
    solves = 1 + N_SOURCES
    ms_total, value = replica_aggregate(ms_local, 1, solves * m * K, dev)
    if world > 1:  # the whole job's time is the slowest rank's; every rank solved the same problems together
        tt = torch.tensor([ms_local], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_total = float(tt.item())
        value = solves * m * K / (ms_total * 1e-3) / 1e9
    pr_sweeps = statistics.mean(s[0] for s in sweeps)
    bf_sweeps = statistics.mean(x for s in sweeps for x in s[1:])
    step_bytes = algorithmic_bytes(n, m, "pr") * pr_sweeps + algorithmic_bytes(n, m, "bf8") * bf_sweeps * N_SOURCES
    per_gpu = step_bytes * K / (ms_total * 1e-3) / 1e9 / world
    peak, peak_kind = _peaks()
    out = {"metric": METRIC, "value": round(value, 3), "unit": "GTEPS", "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": round(ms_total / K, 3), "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None, "dtype": "f32/u32",
           "data": "synthetic (seeded RMAT stand-in for the GAP Kron graph)",
           "config": {"workload": f"rmat{SCALE}: pagerank + sssp x{N_SOURCES}, synchronous, rows split over "
                                  f"{world} GPU(s) (Sec. III-A blocks at GPU granularity)",
                      "n": n, "m": m, "parallelism": f"rows x{world}", "sweeps": {"pagerank": pr_sweeps,
                                                                                  "sssp": bf_sweeps},
                      "l2": "inputs larger than L2 (CSR + one-byte weights 0.34 GB)", "graph_gen_s": round(gen_s, 2)},
           "roofline": {"bound": "hbm", "kernel": "sweep_warp_kernel<*,SYNC> (row range)", "achieved": round(per_gpu, 1),
                        "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(per_gpu / peak, 4),
                        "per": "GPU", "traffic": None},
           # per step: PageRank's state conversions, each sweep's row-range kernel and its sums copy
           "clocks": clk, "gpu_launches": int(K * (2 + 2 * pr_sweeps + 2 * bf_sweeps * N_SOURCES)), "e2e": None}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dag", choices=["dag", "reference"])
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the nvidia-smi clock samples of the timed region in this file (rank-suffixed)")
    ap.add_argument("--quick", dest="extras", action="store_false",
                    help="skip the variant table, the adjoint and the batched measurements")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "rows"],
                    help="with several GPUs: independent replicas of the step (default) or one step with the rows "
                         "of the graph split over the GPUs")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.shard == "rows":
        run_gpu_rowshard(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
