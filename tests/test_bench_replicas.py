"""The N > 1 host logic of bench.py (replicas: barrier, max over ranks,
whole-job rate) with two gloo processes on CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, l = bench.replica_env()
    dist = bench.init_replicas(w, l, backend="gloo")
    dist.barrier()
    ms = 100.0 + 25.0 * r          # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, dist, device="cpu")
    rate = bench.whole_job_rate(1000, w, slowest * 1e-3)
    out[r] = (w, r, slowest, rate)
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        w, rr, slowest, rate = res[r]
        assert (w, rr) == (2, r)
        assert slowest == 125.0                      # max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 1000 / 0.125)  # all ranks' units / slowest time


def test_single_process_defaults(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("LOCAL_RANK", raising=False)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_env() == (1, 0, 0)
    assert bench.init_replicas(1, 0) is None
    assert bench.max_over_ranks(3.5, None) == 3.5
