"""Host-side arithmetic of the benchmark's roofline figures (no GPU): the
algorithmic bytes per sweep and per frontier launch, and the recorded-traffic
lookup (scaling by sweeps or by edges run, null once the kernel sources no
longer match the recorded hash)."""
import os

import pytest

import bench


def test_algorithmic_bytes_by_hand():
    n, m = 10, 100
    # rowptr 4(n+1) + own old + new value 8n (+ out-degree 4n for PageRank), colidx 4m + weights
    assert bench.algorithmic_bytes(n, m, "pr") == 44 + 80 + 40 + 4 * 100
    assert bench.algorithmic_bytes(n, m, "bf") == 44 + 80 + 8 * 100
    assert bench.algorithmic_bytes(n, m, "bf8") == 44 + 80 + 5 * 100
    # frontier launch: per-edge part over the edges run, per-vertex part left to the caller
    assert bench.algorithmic_bytes(n, m, "bf8", edges=37) == (5 * 37, 44 + 80)


def _record(tmp_path, digest):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "sweep_traffic.txt").write_text(
        "# comment: ignored\n"
        f"sweep_source_sha256: {digest}\n"
        f"sweep_tma_kernel<BF8> rmat{bench.SCALE} dram_bytes_per_sweep: 1000\n"
        f"sweep_tma_kernel<BF8,frontier> rmat{bench.SCALE} dram_bytes_per_edge_run: 2.5\n")


def test_recorded_traffic_scales_by_sweeps_and_edges(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "abc")
    _record(tmp_path, "abc")
    assert bench._recorded_traffic("sweep_tma_kernel<BF8>", 7) == 7000
    assert bench._recorded_traffic("sweep_tma_kernel<BF8,frontier>", 11, edges=400) == 1000
    assert bench._recorded_traffic("sweep_tma_kernel<PR>", 3) is None  # not recorded


def test_recorded_traffic_is_null_after_a_source_change(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "new")
    _record(tmp_path, "old")
    assert bench._recorded_traffic("sweep_tma_kernel<BF8>", 7) is None


def test_committed_record_parses():
    path = os.path.join(bench.ROOT, "profiles", "sweep_traffic.txt")
    keys = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#") and ":" in line:
                k, v = line.split(":", 1)
                keys[k.strip()] = v.strip()
    assert len(keys["sweep_source_sha256"]) == 64
    figures = {k: float(v) for k, v in keys.items() if k != "sweep_source_sha256"}
    assert figures and all(v > 0 for v in figures.values())
    assert all(k.endswith((f"rmat{bench.SCALE} dram_bytes_per_sweep", f"rmat{bench.SCALE} dram_bytes_per_edge_run"))
               for k in figures)
    # at least one frontier kernel has a per-edge figure (the step's Bellman-Ford runs one)
    assert any(k.endswith(f"rmat{bench.SCALE} dram_bytes_per_edge_run") and float(v) > 0 for k, v in keys.items())
    if keys["sweep_source_sha256"] != bench.sweep_source_hash():
        pytest.skip("kernel sources changed since the capture: the bench reports traffic as null")


def test_source_hash_covers_every_sweep_kernel_source():
    # a recorded traffic figure must go null when any file of a timed sweep kernel changes
    csrc = os.path.join(bench.ROOT, "paper_2110_01409_gb300", "csrc")
    sweep_files = {f for f in os.listdir(csrc) if f.startswith("sweep") and f.endswith((".cu", ".cuh"))}
    assert sweep_files <= set(bench.SWEEP_SOURCES)
    assert {"sweep_common.cuh", "dag_internal.cuh"} <= set(bench.SWEEP_SOURCES)


def test_kernel_names_of_the_steps_choices_have_recorded_keys():
    # the tuner's choices for the step (and the delayed rows) name kernels that the record holds
    path = os.path.join(bench.ROOT, "profiles", "sweep_traffic.txt")
    with open(path) as f:
        keys = {line.split(" rmat")[0] for line in f if line.strip() and not line.startswith(("#", "sweep_source"))}
    assert bench.kernel_name("BF8", "async", 0, "ordered+cached+frontier", 7) in keys
    assert bench.kernel_name("BF8", "delayed", 0, "warp+cached+frontier", 7) in keys
    assert bench.kernel_name("PR", "async", 0, "ordered+cached", 11) in keys
    assert bench.kernel_name("PR", "delayed", 256, "warp+cached", 7) in keys
    assert bench.kernel_name("BF8", "delayed", 256, "warp+cached", 7) in keys
    # the CTA-tile names
    assert bench.kernel_name("BF8", "async", 0, "cached+frontier") == "sweep_tma_kernel<BF8,frontier>"
    assert bench.kernel_name("PR", "delayed", 32, "refresh") == "sweep_kernel<PR,DELAYED>"
