"""The autotuner's host logic without a GPU: candidate expansion, worker
fractions, failed candidates, the choice of the fastest, the cache and the
locality cutoff. The timed solve (`_run`) and the plan are stand-ins."""
import numpy as np
import pytest
import torch

from paper_2110_01409_gb300 import autotune as A
from paper_2110_01409_gb300 import dag


class FakePlan:
    def __init__(self, n=1000, m=5000, seed=0):
        rng = np.random.default_rng(seed)
        self.n, self.m = n, m
        self.rowptr = torch.from_numpy(np.sort(rng.integers(0, m, n + 1)).astype(np.int32))
        self.colidx = torch.from_numpy(rng.integers(0, n, m).astype(np.int32))
        self.caps = []
        self.tiles = []

    def workers(self, variant="async", delta=0):
        return 608

    def set_worker_cap(self, cap):
        self.caps.append(cap)

    def set_warp_tile(self, ipt):
        self.tiles.append(ipt)


def _fake_run(times, calls, fail=()):
    def run(plan, algo, variant, delta, reads, kw):
        cap = plan.caps[-1]
        calls.append((variant, delta, reads, cap))
        if (variant, delta, reads) in fail:
            raise dag.DagError(-1, "does not fit")
        return times[(variant, delta, reads, cap)], {"iters": 3}
    return run


@pytest.fixture(autouse=True)
def _no_device(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def test_norm_fills_the_read_path_and_warp_tile():
    assert A._norm(("async", 0)) == ("async", 0, "refresh", 7)
    assert A._norm(("async", "0", "own_l1")) == ("async", 0, "own_l1", 7)
    assert A._norm(("async", 0, "warp+cached", 11)) == ("async", 0, "warp+cached", 11)
    with pytest.raises(ValueError):
        A._norm(("async", 0, "warp", 9))  # no such warp tile is built


def test_fingerprint_depends_on_the_graph():
    a, b = FakePlan(seed=1), FakePlan(seed=2)
    assert A.fingerprint(a) == A.fingerprint(FakePlan(seed=1))
    assert A.fingerprint(a) != A.fingerprint(b)
    assert A.fingerprint(a).startswith("n1000_m5000_")


def test_tune_picks_the_fastest_over_candidates_and_worker_fractions(monkeypatch):
    plan = FakePlan()
    cands = [("async", 0), ("delayed", 32), ("async", 0, "own_l1")]
    times = {}
    for i, (v, d, r, _) in enumerate(A._norm(c) for c in cands):
        times[(v, d, r, 0)] = 5.0 + i
        times[(v, d, r, 304)] = 3.5 if (v, d) == ("delayed", 32) else 9.0
    calls = []
    monkeypatch.setattr(A, "_run", _fake_run(times, calls))
    ch = A.tune(plan, "pagerank", candidates=cands, worker_fractions=[1.0, 0.5], trials=2, cache=None)
    assert (ch["variant"], ch["delta"], ch["reads"], ch["workers"]) == ("delayed", 32, "refresh", 304)
    assert ch["ms"] == 3.5 and plan.caps[-1] == 304  # the plan is left at the chosen cap
    assert len(calls) == 2 * 3 * 2  # fractions x candidates x trials
    assert len(ch["candidates"]) == 6


def test_a_failing_candidate_is_recorded_not_chosen(monkeypatch):
    plan = FakePlan()
    times = {("async", 0, "refresh", 0): 3.0, ("delayed", 4096, "refresh", 0): 1.0}
    monkeypatch.setattr(A, "_run", _fake_run(times, [], fail={("delayed", 4096, "refresh")}))
    ch = A.tune(plan, "sssp", candidates=[("async", 0), ("delayed", 4096)], worker_fractions=[1.0], cache=None)
    assert ch["variant"] == "async"
    assert any("error" in r and r["delta"] == 4096 for r in ch["candidates"])


def test_cache_hit_skips_timing_and_sets_the_cap(monkeypatch, tmp_path):
    plan = FakePlan()
    cache = str(tmp_path / "tune.json")
    times = {("async", 0, "refresh", 0): 2.0, ("async", 0, "refresh", 304): 1.0}
    calls = []
    monkeypatch.setattr(A, "_run", _fake_run(times, calls))
    first = A.tune(plan, "pagerank", candidates=[("async", 0)], cache=cache)
    n_calls = len(calls)
    plan2 = FakePlan()  # same graph, new plan
    again = A.tune(plan2, "pagerank", candidates=[("async", 0)], cache=cache)
    assert len(calls) == n_calls  # nothing timed
    assert again == first and plan2.caps == [304]
    # another algorithm or batch width is another key
    A.tune(plan, "sssp", candidates=[("async", 0)], cache=cache)
    assert len(calls) > n_calls


def test_locality_cutoff_drops_the_buffered_candidates(monkeypatch):
    plan = FakePlan()
    times = {(v, d, "refresh", 0): t for (v, d), t in [(("async", 0), 2.0), (("delayed", 32), 1.0)]}
    calls = []
    monkeypatch.setattr(A, "_run", _fake_run(times, calls))
    monkeypatch.setattr(dag, "access_matrix", lambda plan, workers: torch.eye(4, dtype=torch.int64) * 9 + 1)
    ch = A.tune(plan, "pagerank", candidates=[("async", 0), ("delayed", 32)], worker_fractions=[1.0],
                cache=None, locality_cutoff=0.5)
    assert {c[0] for c in calls} == {"async"} and ch["variant"] == "async"
    assert ch["locality"]["diag_share"] == pytest.approx(40 / 52)
    calls.clear()
    ch = A.tune(plan, "pagerank", candidates=[("async", 0), ("delayed", 32)], worker_fractions=[1.0],
                cache=None, locality_cutoff=0.9)
    assert ch["variant"] == "delayed"  # below the cutoff every candidate is timed


def test_warp_candidates_set_their_tile_and_the_choice_keeps_it(monkeypatch):
    plan = FakePlan()
    cands = [("async", 0, "warp+cached", 5), ("async", 0, "warp+cached", 11), ("sync", 0)]
    times = {("async", 0, "warp+cached", 0): 2.0, ("sync", 0, "refresh", 0): 4.0}
    seen = []

    def run(plan_, algo, variant, delta, reads, kw):
        seen.append((reads, plan_.tiles[-1] if reads.startswith("warp") else None))
        ms = 1.0 if (reads, plan_.tiles[-1]) == ("warp+cached", 11) else times[(variant, delta, reads, 0)]
        return ms, {"iters": 3}

    monkeypatch.setattr(A, "_run", run)
    ch = A.tune(plan, "pagerank", candidates=cands, worker_fractions=[1.0], trials=1, cache=None)
    assert ("warp+cached", 5) in seen and ("warp+cached", 11) in seen
    assert (ch["reads"], ch["warp_tile"]) == ("warp+cached", 11) and plan.tiles[-1] == 11


def test_ordered_candidates_set_their_tile_too(monkeypatch):
    # ordered warp sweeps run warp tiles: each candidate must run at its own shape, even after a
    # warp-worker candidate left the plan at another one
    plan = FakePlan()
    cands = [("async", 0, "warp+cached", 11), ("async", 0, "ordered+cached", 7), ("async", 0, "ordered+cached", 11)]
    seen = []

    def run(plan_, algo, variant, delta, reads, kw):
        seen.append((reads, plan_.tiles[-1]))
        return {("ordered+cached", 7): 1.0}.get((reads, plan_.tiles[-1]), 2.0), {"iters": 3}

    monkeypatch.setattr(A, "_run", run)
    ch = A.tune(plan, "pagerank", candidates=cands, worker_fractions=[1.0], trials=1, cache=None)
    assert seen == [("warp+cached", 11), ("ordered+cached", 7), ("ordered+cached", 11)]
    assert (ch["reads"], ch["warp_tile"]) == ("ordered+cached", 7) and plan.tiles[-1] == 7
    assert dag.uses_warp_tile("ordered") and dag.uses_warp_tile("warp+cached") and not dag.uses_warp_tile("own_l1")
