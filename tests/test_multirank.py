"""The replicated multi-GPU path of bench.py on CPU ranks (gloo, world size 2):
the whole-job rate uses the slowest rank's time and counts every rank's
points; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]  # rank 1 is the slow one
    ms, value = bench.job_rate(local_ms, 5, 1000, world, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        shared = mgr.dict()
        mp.spawn(_worker, args=(2, port, shared), nprocs=2, join=True)
        out = dict(shared)
    for r in range(2):
        ms, value = out[r]
        assert ms == pytest.approx(250.0 / 5)
        assert value == pytest.approx(2 * 1000 / (50.0 / 1e3))


def test_job_rate_single_rank():
    import bench
    ms, value = bench.job_rate(80.0, 4, 500, 1, None, "cpu")
    assert ms == 20.0 and value == pytest.approx(500 / 0.02)


def test_reference_arm_only_on_rank0(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        n, steps, warmup = 2000, 1, 0
    bench.run_reference(A())  # returns at once on rank 1, no oracle run
    assert capsys.readouterr().out == ""
