"""bench.py's multi-GPU arithmetic (replicas only: every rank runs its own copy
of the workload), exercised with two gloo ranks on the CPU: the time taken is
the slowest rank's and the throughput counts every rank's units."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slow replica
    worst = bench.max_over_ranks(dist, ms, "cpu")
    out[rank] = (worst, bench.replica_value(1000, world, worst))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = 29500 + (os.getpid() % 2000)
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        worst, value = out[r]
        assert worst == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.replica_value(10, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload = "large"; steps = 1; warmup = 0; gpus = 2
    assert bench.run_reference(A()) == 0
