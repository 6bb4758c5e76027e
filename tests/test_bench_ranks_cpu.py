"""bench.py with several ranks (one replica per GPU under torchrun): the time
of a timed region is the slowest rank's on every rank, and the reference arm
runs on rank 0 only.  Two gloo ranks on the CPU (spawned processes)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        out[rank] = bench._slowest(10.0 + 5.0 * rank, ws, "cpu")
    finally:
        dist.destroy_process_group()


def test_timed_region_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_one_rank_keeps_its_own_time():
    import bench
    assert bench._slowest(12.5, 1, "cpu") == 12.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(None) == 0  # returns before any work or argument
