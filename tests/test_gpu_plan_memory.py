"""Plans built and destroyed in turn (the end-to-end path: a plan per call).

Plans take their device memory from a pool the library keeps per device, which
holds up to 4 GiB of what destroyed plans held for the next plans. Checked
here: plans of graphs of different sizes, each destroyed before the next is
built and each running the frontier and ordered forms (whose maps and
look-back arrays are built on first use), give distances bit-exact against
Dijkstra and ranks within the PageRank tests' L1 bound of the fp64 fixed
point, every time; and the device memory that the churn leaves in use stays
within the pool's bound.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_01409_gb300.inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dag():
    from paper_2110_01409_gb300 import build, dag as D

    build.build()
    assert torch.cuda.is_available()
    return D


def test_plan_churn_results_and_memory(dag):
    graphs = [I.rmat(s, 16, seed=30 + s) for s in (15, 12, 16, 13, 15)]
    refs = {}
    for g in graphs:
        w = I.weights_u32(g, 4).astype(np.uint8)
        src = int(I.sources(g, 1, seed=5)[0])
        key = g.name
        if key not in refs:
            refs[key] = (oracle.dijkstra(g, w.astype(np.uint32), src), oracle.pagerank_fixed_point(g, 0.85))
        d_ref, r_ref = refs[key]
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for rep in range(2):
            plan = dag.Plan.from_graph(g, "cuda")
            d, st = dag.sssp(plan, src, torch.from_numpy(w).cuda(), "async", 0, None, reads="ordered+cached+frontier")
            assert st["converged"]
            assert np.array_equal(d.cpu().numpy().view(np.uint32), d_ref), (key, rep)
            r, st = dag.pagerank(plan, 0.85, 1e-6, "async", 0, 1000, reads="ordered+cached")
            assert st["converged"]
            assert float(np.abs(r.cpu().numpy().astype(np.float64) - r_ref).sum()) <= 1e-5, (key, rep)
            plan.close()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        # what the destroyed plans left mapped is the pool's keep (4 GiB) at most
        assert free0 - free1 <= (4 << 30) + (64 << 20), (key, free0 - free1)
