"""The Python binding fails loudly instead of falling back to the CPU: host
tensors and wrong shapes are refused before any library call, and a missing
libdag.so is an ImportError (no GPU needed)."""
import numpy as np
import pytest
import torch

from paper_2110_01409_gb300 import dag
import paper_2110_01409_gb300.inputs as I


def test_plan_refuses_host_tensors():
    g = I.rmat(6, 4, seed=1)
    with pytest.raises(ValueError, match="CUDA"):
        dag.Plan(torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx))


@pytest.mark.parametrize("bad", ["host", "dtype", "size", "strided"])
def test_device_argument_checks(bad):
    t = torch.zeros(8, dtype=torch.int32)
    if bad == "dtype":
        t = t.float()
    elif bad == "size":
        t = t[:7]
    elif bad == "strided":
        t = torch.zeros(16, dtype=torch.int32)[::2]
    with pytest.raises(ValueError):
        dag._dev(t, torch.int32, 8, "x")


def test_missing_library_is_an_import_error(monkeypatch, tmp_path):
    monkeypatch.setattr(dag, "LIB_PATH", str(tmp_path / "libdag.so"))
    monkeypatch.setattr(dag, "_lib", None)
    with pytest.raises(ImportError, match="libdag.so not found"):
        dag.lib()


def test_variant_and_read_mode_names():
    assert dag._variant("sync") == 0 and dag._variant("async") == 1 and dag._variant("delayed") == 2
    # read paths are disjoint bit flags of the ABI, combinations included
    for name, flags in dag.READ_MODES.items():
        parts = name.split("+")
        if len(parts) > 1:
            assert flags == sum(dag.READ_MODES[p] for p in parts), name
    assert dag.READ_MODES["refresh"] == 0


@pytest.mark.parametrize("bad", ["host", "int64"])
def test_noalloc_refuses_bad_colidx_before_any_library_call(bad, monkeypatch):
    # rowptr and out would pass; a host or int64 colidx must be refused in Python,
    # before its address could reach the kernels
    calls = []
    monkeypatch.setattr(dag, "lib", lambda: calls.append(1))
    rowptr = torch.zeros(9, dtype=torch.int32)
    colidx = torch.zeros(4, dtype=torch.int64 if bad == "int64" else torch.int32)
    monkeypatch.setattr(dag, "_dev", _dev_accepting(rowptr))
    with pytest.raises(ValueError, match="colidx"):
        dag.pagerank_noalloc(rowptr, colidx, out=torch.zeros(8))
    assert not calls


def _dev_accepting(rowptr):
    """_dev that lets the (host) rowptr and output through, so that the colidx
    check is the one that fails."""
    real = dag._dev

    def check(t, dtype, n, name):
        if name in ("rowptr", "out", "teleport"):
            return t
        return real(t, dtype, n, name)

    return check


class _FakePlan:
    def __init__(self, n, m):
        self.n, self.m, self.h = n, m, None


@pytest.mark.parametrize("bad", ["rank", "s", "c", "val", "val_out"])
def test_adjoint_refuses_host_tensors_before_any_library_call(bad, monkeypatch):
    # every array of the adjoint reaches the kernels as a device address: a host (or mis-sized) one is
    # refused in Python first
    calls = []
    monkeypatch.setattr(dag, "lib", lambda: calls.append(1))
    n, m = 8, 12
    real = dag._dev

    def check(t, dtype, k, name):  # the other arrays pass as if they were on the device
        return real(t, dtype, k, name) if name == bad else t

    monkeypatch.setattr(dag, "_dev", check)
    args = dict(val=torch.zeros(m), val_out=torch.zeros(m), s=torch.zeros(n), rank=torch.zeros(n),
                c=torch.zeros(n))
    with pytest.raises(ValueError, match=bad):
        dag.pagerank_adjoint(_FakePlan(n, m), _FakePlan(n, m), **args)
    assert not calls


@pytest.mark.parametrize("which", ["ppr", "sssp"])
def test_batched_refuses_a_host_output_before_any_library_call(which, monkeypatch):
    calls = []
    monkeypatch.setattr(dag, "lib", lambda: calls.append(1))
    n, m, B = 8, 12, 4
    real = dag._dev
    monkeypatch.setattr(dag, "_dev", lambda t, dtype, k, name: real(t, dtype, k, name) if name == "out" else t)
    plan = _FakePlan(n, m)
    with pytest.raises(ValueError, match="out"):
        if which == "ppr":
            dag.ppr_batched(plan, torch.zeros(n, B), out=torch.zeros(n, B))
        else:
            dag.sssp_batched(plan, torch.zeros(B, dtype=torch.int32), torch.zeros(m, dtype=torch.uint8),
                             out=torch.zeros(n, B, dtype=torch.int32))
    assert not calls
