"""The C ABI library builds, loads and exports every symbol include/dag.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "dag.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(dag_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_01409_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("dag_plan_create", "dag_pagerank", "dag_sssp", "dag_ppr_batched", "dag_sssp_batched",
                 "dag_pagerank_adjoint", "dag_transpose", "dag_normalize_weights", "dag_partition",
                 "dag_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu(lib):
    lib.dag_strerror.restype = ctypes.c_char_p
    assert lib.dag_strerror(0) == b"ok"
    assert b"timeout" in lib.dag_strerror(-3)
    assert lib.dag_strerror(12345) == b"unknown error"


def test_binding_lists_match_header():
    from paper_2110_01409_gb300 import dag

    assert sorted(dag.EXPORTS) == _declared()


def test_null_arguments_rejected_on_host(lib):
    # argument checks run before any CUDA call, so they work without a GPU
    lib.dag_plan_create.restype = ctypes.c_int
    assert lib.dag_plan_create(None, 0, None) == -1
    assert lib.dag_pagerank(None, ctypes.c_float(0.85), ctypes.c_double(1e-6), 0, 0, 10, None, None, None, 0,
                            None, None) == -1
