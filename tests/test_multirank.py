"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
renders its own frames (weak scaling, no data-path collective), the job time
is the max over ranks, throughput counts every rank's frames, and only rank 0
runs the reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    frames = [bench.frame_index(k, rank, 32) for k in range(8)]
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    job_ms = bench.max_over_ranks(local_ms, world)
    out[rank] = (frames, job_ms, bench.job_throughput(8, world, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    f0, t0, v0 = out[0]
    f1, t1, v1 = out[1]
    assert t0 == t1 == 150.0
    assert v0 == v1 == pytest.approx(2 * 8 / 0.150)
    assert len(set(f0)) == 8 and len(set(f1)) == 8 and f0 != f1


def test_reference_arm_only_rank0(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        surfels, frames, steps, warmup, gpus, cpu_seconds = 10, 2, 1, 1, 2, 1.0
    # returns immediately on rank 1: no scene, no oracle, no output
    assert bench.run_reference(A()) is None
