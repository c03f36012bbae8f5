"""The multi-rank parts of bench.py on CPU: two gloo ranks agree on the slowest
rank's time, the whole-job value aggregates the ranks' independent patches, and
the reference leg runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    slowest = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)    # rank 1 is the slow one
    out[rank] = (slowest, bench.aggregate_value(world, 1000, slowest))
    bench.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 2 * 1000 / 15e-3)


def test_reference_leg_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus, ref_step_seconds = 1, 3, 2, 1.0
    assert bench.run_reference(A()) == 0
