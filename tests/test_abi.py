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


def test_null_arguments_are_refused_without_a_gpu(lib):
    # every entry point that takes a plan or a CSR refuses a null one with DAG_ERR_INVALID and a
    # message, before touching the device; destroying a null plan is a no-op
    f, d = ctypes.c_float, ctypes.c_double
    N = None
    lib.dag_last_error_message.restype = ctypes.c_char_p
    calls = {
        "dag_plan_create": lambda: lib.dag_plan_create(N, 0, ctypes.byref(ctypes.c_void_p())),
        "dag_plan_out_degree": lambda: lib.dag_plan_out_degree(N, N, N),
        "dag_partition": lambda: lib.dag_partition(N, 4, N),
        "dag_workers": lambda: lib.dag_workers(N, 1, 0, ctypes.byref(ctypes.c_int32())),
        "dag_plan_set_worker_cap": lambda: lib.dag_plan_set_worker_cap(N, 0),
        "dag_plan_set_batched_graph": lambda: lib.dag_plan_set_batched_graph(N, 1),
        "dag_plan_set_warp_tile": lambda: lib.dag_plan_set_warp_tile(N, 7),
        "dag_plan_set_warp_frontier_marks": lambda: lib.dag_plan_set_warp_frontier_marks(N, ctypes.c_float(1.0)),
        "dag_plan_set_batched_wide": lambda: lib.dag_plan_set_batched_wide(N, 1),
        "dag_plan_last_status": lambda: lib.dag_plan_last_status(N, N, N),
        "dag_rank_to_state": lambda: lib.dag_rank_to_state(N, N, N, N, N),
        "dag_state_to_rank": lambda: lib.dag_state_to_rank(N, N, N, N),
        "dag_pagerank_sweep_rows": lambda: lib.dag_pagerank_sweep_rows(N, f(0.85), 0, 1, N, d(1.0), d(0.0), N, N,
                                                                       N, N),
        "dag_sssp_sweep_rows": lambda: lib.dag_sssp_sweep_rows(N, 0, 1, N, N, N, N, N),
        "dag_pagerank": lambda: lib.dag_pagerank(N, f(0.85), d(1e-6), 1, 0, 10, N, N, N, 0, N, N),
        "dag_sssp": lambda: lib.dag_sssp(N, 0, 1, 0, 10, N, N, 0, N, N),
        "dag_sssp_u8": lambda: lib.dag_sssp_u8(N, 0, 1, 0, 10, N, N, 0, N, N),
        "dag_ppr_batched": lambda: lib.dag_ppr_batched(N, f(0.85), d(1e-6), 1, 0, 10, 4, N, N, N, N, N),
        "dag_sssp_batched": lambda: lib.dag_sssp_batched(N, 1, 0, 10, 4, N, N, N, N, N, N),
        "dag_sssp_batched_u8": lambda: lib.dag_sssp_batched_u8(N, 1, 0, 10, 4, N, N, N, N, N, N),
        "dag_transpose": lambda: lib.dag_transpose(N, N, N, N, N),
        "dag_normalize_weights": lambda: lib.dag_normalize_weights(N, N, N, N, N),
        "dag_pagerank_adjoint": lambda: lib.dag_pagerank_adjoint(N, N, f(0.85), d(1e-6), 1, 0, 10, N, N, N, N, N,
                                                                 N, N, N, 0, N, N),
        "dag_pagerank_noalloc": lambda: lib.dag_pagerank_noalloc(N, f(0.85), d(1e-6), 1, 0, 10, N, N, N, N),
        "dag_access_matrix": lambda: lib.dag_access_matrix(N, 4, N, N),
        "dag_debug_skip_barrier_once": lambda: lib.dag_debug_skip_barrier_once(N, 100),
        "dag_debug_stall_staging_once": lambda: lib.dag_debug_stall_staging_once(N, 100),
    }
    for name, call in calls.items():
        assert call() == -1, name
        assert lib.dag_last_error_message(), name
    assert lib.dag_plan_destroy(N) == 0
