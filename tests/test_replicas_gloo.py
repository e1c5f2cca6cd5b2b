"""The multi-GPU path is replicas only: each rank evaluates its own independent
samples, and the ranks share only the timing barrier and the max-over-ranks of
the elapsed time.  These tests run that host logic as two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    total_ms, value = bench.aggregate(100.0 + 50.0 * rank, batch=256, steps=5, dist=dist)
    out[rank] = (total_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # both ranks see the slowest rank's time; the rate counts both ranks' samples
    for r in range(world):
        assert res[r][0] == 150.0
        assert res[r][1] == pytest.approx(world * 256 * 5 / 0.150)


def test_single_process_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(200.0, 256, 5) == (200.0, 256 * 5 / 0.2)


def test_reference_arm_non_zero_rank_exits_quietly(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--config", "grid33"]) == 0
    assert capsys.readouterr().out == ""
