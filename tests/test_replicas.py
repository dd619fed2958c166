"""The benchmark's multi-GPU path is N independent replicas; its only exchange
is the max over ranks of the timed region. Two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        assert b._dist_env()[:2] == (rank, world)
        ms_local = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms, value = b.replica_aggregate(ms_local, world, 1_000_000_000, "cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_take_the_slowest_rank_and_count_every_rank(world):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    slowest = 10.0 + 5.0 * (world - 1)
    for r in range(world):
        ms, value = res[r]
        assert ms == slowest  # every rank reports the same max
        assert value == pytest.approx(world * 1.0 / (slowest * 1e-3))  # GTEPS: world * 1e9 edges over the max


def test_single_rank_needs_no_exchange():
    ms, value = _bench().replica_aggregate(8.0, 1, 2_000_000_000, "cpu")
    assert ms == 8.0 and value == pytest.approx(2.0 / 8e-3)
