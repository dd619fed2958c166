"""Run one solve on a generated graph and print its statistics as JSON.

    python -m paper_2110_01409_gb300.cli --graph rmat --scale 20 --algo sssp --variant delayed --delta 32
    python -m paper_2110_01409_gb300.cli --graph rmat --scale 21 --algo adjoint --variant async --delta 0 \
        --reads warp+cached

Used for single-kernel profiling captures (a small case of the benchmark's
kernels) and for quick experiments from the shell.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import build as B
from . import dag
from . import inputs as I


def make_graph(kind: str, scale: int, seed: int):
    if kind == "rmat":
        return I.rmat(scale, 16, 0.57, 0.19, 0.19, seed=seed)
    if kind == "er":
        return I.erdos_renyi(1 << scale, 16, seed=seed)
    if kind == "banded":
        return I.banded(1 << scale, 15, 1024, 1, seed=seed)
    raise ValueError(kind)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graph", default="rmat", choices=["rmat", "er", "banded"])
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--algo", default="pagerank", choices=["pagerank", "sssp", "sssp8", "adjoint"],
                    help="sssp8: Bellman-Ford with one-byte weights (dag_sssp_u8); adjoint: weighted PageRank "
                         "forward and backward (FP32 weights, 4,096 targets), the same form for both")
    ap.add_argument("--variant", default="delayed", choices=list(dag.VARIANTS))
    ap.add_argument("--delta", type=int, default=256)
    ap.add_argument("--reads", default="refresh", choices=list(dag.READ_MODES))
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--warp-tile", type=int, default=7, help="items per lane of warp tiles (reads warp...)")
    args = ap.parse_args()
    B.build()
    g = make_graph(args.graph, args.scale, args.seed)
    plan = dag.Plan.from_graph(g, "cuda")
    plan.set_warp_tile(args.warp_tile)
    out = []
    model = None
    if args.algo == "adjoint":
        model = dag.WeightedPageRank(plan, d=0.85, tol=args.tol, variant=args.variant, delta=args.delta,
                                     reads=args.reads)
        w_f = torch.from_numpy(I.weights_f32(g, args.seed)).cuda()
        targets, wt = I.adjoint_targets(g.n, 4096, seed=5)
        c = torch.zeros(g.n, dtype=torch.float32, device="cuda")
        c[torch.from_numpy(targets).cuda()] = torch.from_numpy(wt.astype(np.float32)).cuda()
    for _ in range(args.repeat):
        if args.algo == "adjoint":
            r, val, s, st_f = model.forward(w_f)
            _, _, _, st = model.backward(val, s, r, c)
            st = {"forward": st_f, "backward": st}
        elif args.algo == "pagerank":
            _, st = dag.pagerank(plan, 0.85, args.tol, args.variant, args.delta, reads=args.reads)
        else:
            w32 = I.weights_u32(g, args.seed)
            w = torch.from_numpy(w32.astype(np.uint8) if args.algo == "sssp8" else w32.view(np.int32)).cuda()
            src = int(I.sources(g, 1, seed=args.seed)[0])
            _, st = dag.sssp(plan, src, w, args.variant, args.delta, reads=args.reads)
        out.append(st)
    torch.cuda.synchronize()
    print(json.dumps({"graph": args.graph, "scale": args.scale, "n": g.n, "m": g.m, "algo": args.algo,
                      "variant": args.variant, "delta": args.delta, "reads": args.reads, "runs": out}))


if __name__ == "__main__":
    main()
